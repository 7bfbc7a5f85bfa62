// prims.cu -- integer primitives used by the setup phase: device-wide
// exclusive scan, stable LSD radix sort of (key, value) pairs, stream
// compaction and small reductions.  Every result is exact and independent of
// scheduling (integer arithmetic only), which the bit-exact setup relies on.
#include "lamg_internal.cuh"

namespace lamg {

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (values and total must fit in int32).
// Tiles of 1024 threads x 4 items; tile sums are scanned recursively.
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int32_t *__restrict__ out,
                             int32_t *__restrict__ tile_sums, int64_t n) {
    __shared__ int32_t wpart[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        sum += v[i];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t inc = warp_incl_scan(sum);
    if (lane == 31) wpart[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int32_t s = wpart[lane];
        int32_t si = warp_incl_scan(s);
        wpart[lane] = si - s;
        if (lane == 31 && tile_sums) tile_sums[blockIdx.x] = si;
    }
    __syncthreads();
    int32_t run = inc - sum + wpart[wid];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

__global__ void k_scan_add(int32_t *__restrict__ out, const int32_t *__restrict__ tile_offs,
                           int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    const int32_t add = tile_offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; i++)
        if (base + i < n) out[base + i] += add;
}

void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int tiles = ceil_div(n, kScanTile);
    if (tiles == 1) {
        k_scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, nullptr, n);
        LAMG_CHECK_LAUNCH();
        return;
    }
    Tmp<int32_t> sums(tiles, s), offs(tiles, s);
    k_scan_tiles<<<tiles, kScanThreads, 0, s>>>(in, out, sums.get(), n);
    LAMG_CHECK_LAUNCH();
    exclusive_scan_i32(sums.get(), offs.get(), tiles, s);
    k_scan_add<<<tiles, kScanThreads, 0, s>>>(out, offs.get(), n);
    LAMG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.
// Upsweep: per-tile digit histograms (digit-major layout), exclusive scan,
// downsweep: each warp ranks its consecutive sub-tile with __match_any_sync,
// warps are offset by per-warp digit counts, so equal keys keep input order.
// ---------------------------------------------------------------------------

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096
constexpr int kSortWarpTile = 32 * kSortItems;        // 512

template <class K>
__global__ void k_sort_hist(const K *__restrict__ keys, int64_t n, int shift,
                            int32_t *__restrict__ hist, int ntiles) {
    __shared__ int32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(int)((keys[idx] >> shift) & 0xFF)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

template <class K, class V>
__global__ void k_sort_scatter(const K *__restrict__ kin, const V *__restrict__ vin,
                               K *__restrict__ kout, V *__restrict__ vout, int64_t n, int shift,
                               const int32_t *__restrict__ offs, int ntiles) {
    __shared__ int32_t cnt[kSortWarps][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)wid * kSortWarpTile;
    K k[kSortItems];
    V v[kSortItems];
    int32_t pos[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kSortItems; i++) {
        int64_t idx = base + i * 32 + lane;
        bool valid = idx < n;
        unsigned act = __ballot_sync(0xffffffffu, valid);
        pos[i] = -1;
        if (valid) {
            k[i] = kin[idx];
            v[i] = vin[idx];
            int d = (int)((k[i] >> shift) & 0xFF);
            unsigned peers = __match_any_sync(act, d);
            int32_t before = cnt[wid][d];
            pos[i] = before + __popc(peers & lt);
            __syncwarp(act);
            if ((peers & lt) == 0) cnt[wid][d] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int32_t run = 0;
        for (int w = 0; w < kSortWarps; w++) {
            int32_t t = cnt[w][d];
            cnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; i++) {
        if (pos[i] >= 0) {
            int d = (int)((k[i] >> shift) & 0xFF);
            int64_t dst = (int64_t)offs[(int64_t)d * ntiles + blockIdx.x] + cnt[wid][d] + pos[i];
            kout[dst] = k[i];
            vout[dst] = v[i];
        }
    }
}

// Sorts (keys, vals) in place by the low `nbits` bits of the key (stable).
// ktmp/vtmp: scratch of n elements each.
template <class K, class V>
void radix_sort_pairs(K *keys, V *vals, K *ktmp, V *vtmp, int64_t n, int nbits, cudaStream_t s) {
    if (n <= 1 || nbits <= 0) return;
    LAMG_REQUIRE(n < ((int64_t)1 << 31), LAMG_ERR_ARG, "radix sort: too many elements");
    int ntiles = ceil_div(n, kSortTile);
    Tmp<int32_t> hist((size_t)ntiles * 256, s), offs((size_t)ntiles * 256, s);
    K *ka = keys, *kb = ktmp;
    V *va = vals, *vb = vtmp;
    int passes = 0;
    for (int shift = 0; shift < nbits; shift += 8, passes++) {
        k_sort_hist<K><<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, hist.get(), ntiles);
        LAMG_CHECK_LAUNCH();
        exclusive_scan_i32(hist.get(), offs.get(), (int64_t)ntiles * 256, s);
        k_sort_scatter<K, V><<<ntiles, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, offs.get(),
                                                             ntiles);
        LAMG_CHECK_LAUNCH();
        K *t = ka; ka = kb; kb = t;
        V *u = va; va = vb; vb = u;
    }
    if (passes & 1) {
        LAMG_CUDA(cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
        LAMG_CUDA(cudaMemcpyAsync(vals, va, sizeof(V) * n, cudaMemcpyDeviceToDevice, s));
    }
}

template void radix_sort_pairs<uint32_t, int32_t>(uint32_t *, int32_t *, uint32_t *, int32_t *,
                                                  int64_t, int, cudaStream_t);
template void radix_sort_pairs<uint64_t, int32_t>(uint64_t *, int32_t *, uint64_t *, int32_t *,
                                                  int64_t, int, cudaStream_t);
template void radix_sort_pairs<uint64_t, double>(uint64_t *, double *, uint64_t *, double *,
                                                 int64_t, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Compaction and reductions
// ---------------------------------------------------------------------------

__global__ void k_u8_to_i32(const uint8_t *__restrict__ f, int32_t *__restrict__ o, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = f[i] ? 1 : 0;
}

__global__ void k_compact(const uint8_t *__restrict__ f, const int32_t *__restrict__ pos,
                          int32_t *__restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && f[i]) out[pos[i]] = (int32_t)i;
}

// Indices i with flags[i] != 0, in increasing order; returns the count.
int64_t compact_indices(const uint8_t *flags, int32_t *out_idx, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    Tmp<int32_t> f(n + 1, s), pos(n + 1, s);
    k_u8_to_i32<<<ceil_div(n, 256), 256, 0, s>>>(flags, f.get(), n);
    LAMG_CHECK_LAUNCH();
    LAMG_CUDA(cudaMemsetAsync(f.get() + n, 0, sizeof(int32_t), s));
    exclusive_scan_i32(f.get(), pos.get(), n + 1, s);
    int32_t total = read_scalar(pos.get() + n, s);
    k_compact<<<ceil_div(n, 256), 256, 0, s>>>(flags, pos.get(), out_idx, n);
    LAMG_CHECK_LAUNCH();
    return total;
}

__global__ void k_reduce_max(const int32_t *__restrict__ a, int64_t n, int32_t *out) {
    int32_t m = INT32_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, a[i]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

int32_t reduce_max_i32(const int32_t *a, int64_t n, cudaStream_t s) {
    Tmp<int32_t> o(1, s);
    int32_t init = INT32_MIN;
    LAMG_CUDA(cudaMemcpyAsync(o.get(), &init, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    int blocks = std::min(ceil_div(n, 256), 152 * 8);
    if (blocks < 1) blocks = 1;
    k_reduce_max<<<blocks, 256, 0, s>>>(a, n, o.get());
    LAMG_CHECK_LAUNCH();
    return read_scalar(o.get(), s);
}

__global__ void k_count_eq(const int32_t *__restrict__ a, int64_t n, int32_t v,
                           unsigned long long *out) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        c += (a[i] == v);
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

int64_t count_equal_i32(const int32_t *a, int64_t n, int32_t value, cudaStream_t s) {
    Tmp<unsigned long long> o(1, s);
    LAMG_CUDA(cudaMemsetAsync(o.get(), 0, sizeof(unsigned long long), s));
    int blocks = std::min(ceil_div(n, 256), 152 * 8);
    if (blocks < 1) blocks = 1;
    k_count_eq<<<blocks, 256, 0, s>>>(a, n, value, o.get());
    LAMG_CHECK_LAUNCH();
    return (int64_t)read_scalar(o.get(), s);
}

}  // namespace lamg
