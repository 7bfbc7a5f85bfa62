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
// The cycle itself runs in the cycle engine (cycle.cu): one persistent
// cooperative kernel per cycle or refinement step.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "solve_rows.cuh"

namespace lamg {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRedBlocksMax = 1024;  // reduction grid: 4 blocks per SM, at most this many
constexpr int kRedThreads = 256;
constexpr int64_t kTailWork32 = 2048;   // entries of a colour that the single-block sweep takes (FP32)
constexpr int64_t kTailWork64 = 512;    // same for FP64 (one SM's FP64 rate is low on this GPU)
constexpr int64_t kSBWork32 = 16384, kSBWork64 = 16384;

int64_t sb_work(const lamg_options &o, int prec) {
    const int32_t v = prec == 1 ? o.sb_work32 : o.sb_work64;
    return v > 0 ? v : (prec == 1 ? kSBWork32 : kSBWork64);
}
int64_t tail_work(const lamg_options &o, int prec) {
    const int32_t v = prec == 1 ? o.tail_work32 : o.tail_work64;
    return v > 0 ? v : (prec == 1 ? kTailWork32 : kTailWork64);
}

// blocks of the two-pass reductions: 4 per SM of the current device
static int red_blocks() {
    int dev = 0, sms = 0;
    LAMG_CUDA(cudaGetDevice(&dev));
    LAMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return std::max(1, std::min(kRedBlocksMax, 4 * sms));
}

// scratch layout (doubles)
enum {
    SC_PART = 0,                     // up to kRedBlocksMax * 8 partial sums
    SC_ALPHA = kRedBlocksMax * 8,    // recombination coefficients per level (2 each)
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
// With several components K (a union of graphs), M = A + sum_K 1_K 1_K^T / n_K:
// comp[i] is the component of row i and inv[k] = 1 / n_k (comp == NULL: one).
__global__ void k_dense_assemble(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 const double *__restrict__ w, double *__restrict__ G,
                                 const int32_t *__restrict__ comp, const double *__restrict__ inv) {
    // G is n x 2n, row-major: [M | I]
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 2 * n) return;
    const int32_t i = (int32_t)(q / (2 * n)), j = (int32_t)(q % (2 * n));
    double v;
    if (j >= n) {
        v = (j - n == i) ? 1.0 : 0.0;
    } else {
        v = comp ? (comp[i] == comp[j] ? inv[comp[i]] : 0.0) : 1.0 / (double)n;
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

// Tail colours of a level: the longest suffix of colours that each hold at most
// kTailRows rows (and together at most kTailMax rows), when it has at least
// kTailMinColours colours.  On power-law levels these are the hubs, which
// need many colours among themselves.  Builds the tail block's local CSR
// (entries whose column is also a tail row) and the full weighted degrees.
constexpr int32_t kTailRows = 64, kTailMax = 4096, kTailMinColours = 4;

static void build_tail(SolveLevel &V, int ncol, cudaStream_t s) {
    V.tc0 = -1;
    V.tn = 0;
    const int32_t n = V.n;
    if (ncol < kTailMinColours + 1) return;
    auto rows = [&](int c) { return V.cb[4 * c + 3] - V.cb[4 * c]; };
    int c0 = ncol;
    while (c0 > 1 && rows(c0 - 1) <= kTailRows && n - V.cb[4 * (c0 - 1)] <= kTailMax) c0--;
    if (ncol - c0 < kTailMinColours) return;
    const int32_t t0 = V.cb[4 * c0], tn = n - t0;
    std::vector<int32_t> hrp(tn + 1);
    LAMG_CUDA(cudaMemcpyAsync(hrp.data(), V.rp.get() + t0, sizeof(int32_t) * (tn + 1), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    const int64_t e0 = hrp[0], ne = (int64_t)hrp[tn] - e0;
    std::vector<int32_t> hcol(ne);
    std::vector<double> hw(ne);
    if (ne) {
        LAMG_CUDA(cudaMemcpyAsync(hcol.data(), V.col.get() + e0, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaMemcpyAsync(hw.data(), V.w64.get() + e0, sizeof(double) * ne, cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaStreamSynchronize(s));
    }
    std::vector<int32_t> trp(tn + 1, 0), tcol, tcb(ncol - c0 + 1);
    std::vector<double> tw, deg(tn);
    std::vector<float> tw32, deg32(tn);
    for (int32_t i = 0; i < tn; i++) {
        double d = 0.0;
        float d32 = 0.f;
        for (int64_t k = hrp[i] - e0; k < hrp[i + 1] - e0; k++) {
            d += hw[k];
            d32 += (float)hw[k];
            if (hcol[k] >= t0) {
                tcol.push_back(hcol[k] - t0);
                tw.push_back(hw[k]);
                tw32.push_back((float)hw[k]);
            }
        }
        deg[i] = d;
        deg32[i] = d32;
        trp[i + 1] = (int32_t)tcol.size();
    }
    for (int c = c0; c <= ncol; c++) tcb[c - c0] = (c < ncol ? V.cb[4 * c] : n) - t0;
    // chunks of kTailChunk local entries: a tail colour step spreads its rows' chunks over all warps
    std::vector<int32_t> trq(tn + 1, 0);
    for (int32_t i = 0; i < tn; i++) trq[i + 1] = trq[i] + (trp[i + 1] - trp[i] + kTailChunk - 1) / kTailChunk;
    int32_t maxq = 0;
    for (int c = 0; c + 1 < (int)tcb.size(); c++) maxq = std::max(maxq, trq[tcb[c + 1]] - trq[tcb[c]]);
    V.tmaxq = maxq;
    V.trq.alloc(tn + 1);
    LAMG_CUDA(cudaMemcpyAsync(V.trq.get(), trq.data(), sizeof(int32_t) * (tn + 1), cudaMemcpyHostToDevice, s));
    V.tc0 = c0;
    V.tt0 = t0;
    V.tn = tn;
    V.tnc = ncol - c0;
    V.tnnz = (int64_t)tcol.size();
    V.trp.alloc(tn + 1);
    V.tcb.alloc(tcb.size());
    V.tcol.alloc(tcol.size());
    V.tw64.alloc(tw.size());
    V.tw32.alloc(tw32.size());
    V.tdeg64.alloc(tn);
    V.tdeg32.alloc(tn);
    LAMG_CUDA(cudaMemcpyAsync(V.trp.get(), trp.data(), sizeof(int32_t) * (tn + 1), cudaMemcpyHostToDevice, s));
    LAMG_CUDA(cudaMemcpyAsync(V.tcb.get(), tcb.data(), sizeof(int32_t) * tcb.size(), cudaMemcpyHostToDevice, s));
    if (!tcol.empty()) {
        LAMG_CUDA(cudaMemcpyAsync(V.tcol.get(), tcol.data(), sizeof(int32_t) * tcol.size(), cudaMemcpyHostToDevice, s));
        LAMG_CUDA(cudaMemcpyAsync(V.tw64.get(), tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice, s));
        LAMG_CUDA(cudaMemcpyAsync(V.tw32.get(), tw32.data(), sizeof(float) * tw32.size(), cudaMemcpyHostToDevice, s));
    }
    LAMG_CUDA(cudaMemcpyAsync(V.tdeg64.get(), deg.data(), sizeof(double) * tn, cudaMemcpyHostToDevice, s));
    LAMG_CUDA(cudaMemcpyAsync(V.tdeg32.get(), deg32.data(), sizeof(float) * tn, cudaMemcpyHostToDevice, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
}

// A level followed by elimination (Sec. 3.2): the permuted coarse id of each
// permuted row (-1 for an eliminated row) and, for the eliminated rows, a_ii
// summed over the row in entry order (degree <= 4).
__global__ void k_elim_layout(int32_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ cidx,
                              const int32_t *__restrict__ iperm_c, const int32_t *__restrict__ rp,
                              const double *__restrict__ w64, const float *__restrict__ w32,
                              int32_t *__restrict__ ecx, double *__restrict__ ed64, float *__restrict__ ed32) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t c = cidx[perm[i]];
    ecx[i] = c < 0 ? -1 : iperm_c[c];
    double d = 0.0;
    float d32 = 0.f;
    if (c < 0)
        for (int32_t j = rp[i]; j < rp[i + 1]; j++) { d += w64[j]; d32 += w32[j]; }
    ed64[i] = d;
    ed32[i] = d32;
}

// Sliced ELL of the thread-tier rows of a level (see SolveLevel): slices of 32
// consecutive rows within each colour's thread-tier range.
__global__ void k_sell_pairs(int32_t nsl, const int4 *__restrict__ sl, const int32_t *__restrict__ rp,
                             int32_t *__restrict__ pairs) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsl) return;
    const int4 m = sl[k];
    int32_t w = 0;
    for (int32_t i = m.x; i < m.x + m.y; i++) w = max(w, rp[i + 1] - rp[i]);
    pairs[k] = (w + 1) >> 1;
}
__global__ void k_sell_offsets(int32_t nsl, const int32_t *__restrict__ pairs, const int32_t *__restrict__ first,
                               int4 *__restrict__ sl) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsl) return;
    sl[k].z = pairs[k];
    sl[k].w = first[k];
}
// one thread per (slice, lane); lanes past the slice's rows get the padding entry
// of its first row
__global__ void k_sell_fill(int32_t nsl, const int4 *__restrict__ sl, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ col, const float *__restrict__ w32,
                            const double *__restrict__ w64, uint4 *__restrict__ ell32, int2 *__restrict__ ellc,
                            double2 *__restrict__ ellw) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nsl * 32) return;
    const int32_t k = (int32_t)(t >> 5), lane = (int32_t)(t & 31);
    const int4 m = sl[k];
    const int32_t i = lane < m.y ? m.x + lane : m.x;
    const int32_t s = lane < m.y ? rp[i] : 0, e = lane < m.y ? rp[i + 1] : 0;
    for (int32_t p = 0; p < m.z; p++) {
        const int32_t j0 = s + 2 * p, j1 = j0 + 1;
        const int32_t c0 = j0 < e ? col[j0] : i, c1 = j1 < e ? col[j1] : i;
        const float a0 = j0 < e ? w32[j0] : 0.0f, a1 = j1 < e ? w32[j1] : 0.0f;
        const double b0 = j0 < e ? w64[j0] : 0.0, b1 = j1 < e ? w64[j1] : 0.0;
        const size_t q = ((size_t)m.w + p) * 32 + lane;
        ell32[q] = make_uint4((unsigned)c0, (unsigned)c1, __float_as_uint(a0), __float_as_uint(a1));
        ellc[q] = make_int2(c0, c1);
        ellw[q] = make_double2(b0, b1);
    }
}

static void build_sell(SolveLevel &V, int ncol, cudaStream_t s) {
    std::vector<int4> hs;
    V.csl.assign(ncol + 1, 0);
    for (int c = 0; c < ncol; c++) {
        const int32_t t0 = V.cb[4 * c], t1 = V.cb[4 * c + 1];
        for (int32_t r = t0; r < t1; r += 32) hs.push_back(make_int4(r, std::min(32, t1 - r), 0, 0));
        V.csl[c + 1] = (int32_t)hs.size();
    }
    V.nsl = (int32_t)hs.size();
    V.csl_dev.alloc(ncol + 1);
    LAMG_CUDA(cudaMemcpyAsync(V.csl_dev.get(), V.csl.data(), sizeof(int32_t) * (ncol + 1), cudaMemcpyHostToDevice, s));
    if (V.nsl == 0) return;
    V.sl.alloc(V.nsl);
    LAMG_CUDA(cudaMemcpyAsync(V.sl.get(), hs.data(), sizeof(int4) * V.nsl, cudaMemcpyHostToDevice, s));
    Tmp<int32_t> pairs(V.nsl + 1, s), first(V.nsl + 1, s);
    LAMG_CUDA(cudaMemsetAsync(pairs.get() + V.nsl, 0, sizeof(int32_t), s));
    k_sell_pairs<<<ceil_div(V.nsl, 256), 256, 0, s>>>(V.nsl, V.sl.get(), V.rp.get(), pairs.get());
    LAMG_CHECK_LAUNCH();
    exclusive_scan_i32(pairs.get(), first.get(), V.nsl + 1, s);
    k_sell_offsets<<<ceil_div(V.nsl, 256), 256, 0, s>>>(V.nsl, pairs.get(), first.get(), V.sl.get());
    LAMG_CHECK_LAUNCH();
    const int64_t total = (int64_t)read_scalar(first.get() + V.nsl, s) * 32;
    LAMG_REQUIRE(total < ((int64_t)1 << 31), LAMG_ERR_OOM, "sliced ELL larger than 2^31 pairs");
    V.ell32.alloc(std::max<int64_t>(total, 1));
    V.ellc.alloc(std::max<int64_t>(total, 1));
    V.ellw64.alloc(std::max<int64_t>(total, 1));
    k_sell_fill<<<ceil_div((int64_t)V.nsl * 32, 256), 256, 0, s>>>(V.nsl, V.sl.get(), V.rp.get(), V.col.get(),
                                                                  V.w32.get(), V.w64.get(), V.ell32.get(),
                                                                  V.ellc.get(), V.ellw64.get());
    LAMG_CHECK_LAUNCH();
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
                const int64_t lim = tail_work(h->opt, p);
                auto small = [&](int c) { return (int64_t)hrp[V.cb[4 * c + 3]] - hrp[V.cb[4 * c]] <= lim; };
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
        build_tail(V, S.ncolours, s);
        build_sell(V, S.ncolours, s);
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
        if (S.elim) {
            V.elim = 1;
            V.ecx.alloc(n);
            V.ed64.alloc(n);
            V.ed32.alloc(n);
            k_elim_layout<<<ceil_div(n, 256), 256, 0, s>>>(n, V.perm.get(), S.cidx.get(), iperm[l + 1].get(),
                                                          V.rp.get(), V.w64.get(), V.w32.get(), V.ecx.get(),
                                                          V.ed64.get(), V.ed32.get());
            LAMG_CHECK_LAUNCH();
            continue;
        }
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
        // connected components of the coarsest graph (host BFS; n <= dense_max)
        std::vector<int32_t> hrp(n + 1), hcol(C.nnz), comp(n, -1);
        LAMG_CUDA(cudaMemcpyAsync(hrp.data(), C.rp.get(), sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s));
        if (C.nnz)
            LAMG_CUDA(cudaMemcpyAsync(hcol.data(), C.col.get(), sizeof(int32_t) * C.nnz, cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaStreamSynchronize(s));
        int32_t ncomp = 0;
        std::vector<int32_t> queue(n);
        std::vector<double> inv;
        for (int32_t s0 = 0; s0 < n; s0++) {
            if (comp[s0] >= 0) continue;
            int32_t head = 0, tail = 0;
            comp[s0] = ncomp;
            queue[tail++] = s0;
            while (head < tail) {
                const int32_t u = queue[head++];
                for (int32_t e = hrp[u]; e < hrp[u + 1]; e++)
                    if (comp[hcol[e]] < 0) { comp[hcol[e]] = ncomp; queue[tail++] = hcol[e]; }
            }
            inv.push_back(1.0 / (double)tail);
            ncomp++;
        }
        Tmp<int32_t> dcomp(ncomp > 1 ? n : 0, s);
        Tmp<double> dinv(ncomp > 1 ? ncomp : 0, s);
        if (ncomp > 1) {
            LAMG_CUDA(cudaMemcpyAsync(dcomp.get(), comp.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
            LAMG_CUDA(cudaMemcpyAsync(dinv.get(), inv.data(), sizeof(double) * ncomp, cudaMemcpyHostToDevice, s));
        }
        k_dense_assemble<<<ceil_div(tot, 256), 256, 0, s>>>(n, C.rp.get(), C.col.get(), C.w64.get(), G.get(),
                                                            ncomp > 1 ? dcomp.get() : nullptr, dinv.get());
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
// Vector helpers (reductions for checks, natural <-> permuted order)
// ---------------------------------------------------------------------------

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

// mode 0: sum, 1: sum of |a|, 2: sum of squares
__global__ void k_partial(int32_t n, const double *__restrict__ a, int mode, double *__restrict__ part) {
    double v = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double t = a[i];
        v += mode == 0 ? t : (mode == 1 ? fabs(t) : t * t);
    }
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void k_finish_sum(const double *__restrict__ part, int nb, double *__restrict__ out) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
    v = block_sum(v);
    if (threadIdx.x == 0) *out = v;
}

static void reduce_to(const double *a, int32_t n, int mode, double *part, double *out, cudaStream_t s) {
    const int nb = red_blocks();
    k_partial<<<nb, kRedThreads, 0, s>>>(n, a, mode, part);
    LAMG_CHECK_LAUNCH();
    k_finish_sum<<<1, 256, 0, s>>>(part, nb, out);
    LAMG_CHECK_LAUNCH();
}

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
// Union of several graphs: level-1 maps for the per-graph projection and norms
// ---------------------------------------------------------------------------

__global__ void k_invert_perm(int32_t n, const int32_t *__restrict__ perm, int32_t *__restrict__ iperm) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) iperm[perm[i]] = i;
}

__global__ void k_gather_i32(int32_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ src,
                             int32_t *__restrict__ dst) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[perm[i]];
}

void graph_ids(int64_t n, const int64_t *gptr_dev, int32_t G, int32_t *gid, cudaStream_t s);

void build_graph_maps(lamg_ctx *h, cudaStream_t s) {
    const int32_t n = h->lv[0].n, G = h->ngraphs;
    h->gptr_d.alloc(G + 1);
    LAMG_CUDA(cudaMemcpyAsync(h->gptr_d.get(), h->gptr.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, s));
    h->gidnat.alloc(n);
    graph_ids(n, h->gptr_d.get(), G, h->gidnat.get(), s);
    h->iperm0.alloc(n);
    k_invert_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, h->lv[0].perm.get(), h->iperm0.get());
    LAMG_CHECK_LAUNCH();
    h->gid0.alloc(n);
    k_gather_i32<<<ceil_div(n, 256), 256, 0, s>>>(n, h->lv[0].perm.get(), h->gidnat.get(), h->gid0.get());
    LAMG_CHECK_LAUNCH();
    h->gsum.alloc(G);
    h->gnorm.alloc(G);
    h->gstat.alloc(3 * (size_t)G);
    LAMG_CUDA(cudaStreamSynchronize(s));
}

// Per graph g (one block per graph, fixed order): over natural ids u in
// [gptr[g], gptr[g+1]) of v[map ? map[u] : u]: out[g] = sum, out[G+g] = sum |.|,
// out[2G+g] = sum of squares.
__global__ void __launch_bounds__(1024) k_graph_stats(int32_t G, const int64_t *__restrict__ gptr,
                                                      const int32_t *__restrict__ map, const double *__restrict__ v,
                                                      double *__restrict__ out) {
    for (int32_t g = blockIdx.x; g < G; g += gridDim.x) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int64_t u = gptr[g] + threadIdx.x; u < gptr[g + 1]; u += blockDim.x) {
            const double t = v[map ? map[u] : u];
            a += t;
            b += fabs(t);
            c += t * t;
        }
        a = block_sum(a);
        b = block_sum(b);
        c = block_sum(c);
        if (threadIdx.x == 0) {
            out[g] = a;
            out[G + g] = b;
            out[2 * G + g] = c;
        }
    }
}

// ---------------------------------------------------------------------------
// Solve drivers
// ---------------------------------------------------------------------------

template <class T>
static void alloc_vecs(lamg_ctx *h, std::vector<LevelVecs<T>> &vv) {
    vv.resize(h->L);
    for (int l = 0; l < h->L; l++) {
        const int32_t n = h->lv[l].n;
        vv[l].x.alloc(n);
        vv[l].b.alloc(n);
        vv[l].r.alloc(n);
        if ((l >= 1 || h->opt.recomb_finest) && l + 1 < h->L) {
            vv[l].xs0.alloc(n); vv[l].xs1.alloc(n);
            vv[l].rs0.alloc(n); vv[l].rs1.alloc(n);
        }
    }
}

static void prepare(lamg_ctx *h) {
    if (h->v64.empty()) alloc_vecs<double>(h, h->v64);
    if (h->v32.empty()) alloc_vecs<float>(h, h->v32);
    if (!h->scratch.get()) h->scratch.alloc(SC_TOTAL);
    if (!h->r64.get()) h->r64.alloc(h->lv[0].n);
    if (!h->host_pinned) LAMG_CUDA(cudaMallocHost((void **)&h->host_pinned, 16 * sizeof(double)));
    engine_prepare(h);
}

void prepare_solve(lamg_ctx *h) { prepare(h); }

// Engine launch of one step with optional CUDA-event timing of the launch.
static void run_step(lamg_ctx *h, int kind, int adaptive, cudaStream_t s) {
    const double mu = adaptive ? h->opt.mu_adaptive : h->opt.mu_flat;
    if (h->prof_on) {
        if (h->prof_ev.size() < 2) {
            for (int k = 0; k < 2; k++) {
                cudaEvent_t e;
                LAMG_CUDA(cudaEventCreate(&e));
                h->prof_ev.push_back(e);
            }
        }
        LAMG_CUDA(cudaEventRecord(h->prof_ev[0], s));
        engine_run(h, kind, adaptive, mu, s);
        LAMG_CUDA(cudaEventRecord(h->prof_ev[1], s));
    } else {
        engine_run(h, kind, adaptive, mu, s);
    }
}

static void after_step(lamg_ctx *h, int kind, cudaStream_t s) {
    if (engine_failed(h, s)) throw Error{LAMG_ERR_TIMEOUT, "cycle engine: grid barrier timed out"};
    if (h->prof_on) {
        float ms = 0.f;
        LAMG_CUDA(cudaEventElapsedTime(&ms, h->prof_ev[0], h->prof_ev[1]));
        h->prof_ms += ms;
        h->prof_count++;
        // algorithmic bytes of one engine launch: the cycles it runs plus the FP64 residual
        const SolveLevel &V = h->lv[0];
        const int64_t res64 = V.nnz * 12 + (int64_t)(V.n + 1) * 4 + (int64_t)V.n * 24;
        if (kind == 1)
            h->prof_bytes = std::max(1, h->opt.ir_inner) * h->last.bytes_per_cycle32 + res64 + (int64_t)V.n * 32;
        else
            h->prof_bytes = h->last.bytes_per_cycle + res64;
    }
}

// sum, ||b||_1 and ||b||_2 of the FP64 right-hand side (zero-sum check, Sec. 1)
static void rhs_norms(lamg_ctx *h, const double *b, cudaStream_t s, double &sum, double &asum, double &nrm) {
    const int32_t n = h->lv[0].n;
    double *part = h->scratch.get() + SC_PART;
    double *out = h->scratch.get() + SC_NORM + 4;
    reduce_to(b, n, 0, part, out, s);
    reduce_to(b, n, 1, part, out + 1, s);
    reduce_to(b, n, 2, part, out + 2, s);
    double hv[3];
    LAMG_CUDA(cudaMemcpyAsync(hv, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    sum = hv[0];
    asum = hv[1];
    nrm = std::sqrt(hv[2]);
}

// ||b - A x||_2 of the permuted FP64 level-1 vectors (r64 <- b - A x)
__global__ void k_res64(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                        const double *__restrict__ w, const double *__restrict__ b, const double *__restrict__ x,
                        double *__restrict__ r) {
    // one warp per row (setup-time check; not on the cycle path)
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= n) return;
    const int32_t i = (int32_t)wg;
    const double xi = x[i];
    double acc = 0.0;
    for (int32_t j = rp[i] + lane; j < rp[i + 1]; j += 32) acc += w[j] * (x[col[j]] - xi);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) r[i] = b[i] + acc;
}

static double resnorm64(lamg_ctx *h, cudaStream_t s) {
    const SolveLevel &V = h->lv[0];
    k_res64<<<ceil_div((int64_t)V.n * 32, 256), 256, 0, s>>>(V.n, V.rp.get(), V.col.get(), V.w64.get(),
                                                            h->v64[0].b.get(), h->v64[0].x.get(), h->r64.get());
    LAMG_CHECK_LAUNCH();
    reduce_to(h->r64.get(), V.n, 2, h->scratch.get() + SC_PART, h->scratch.get() + SC_NORM, s);
    return std::sqrt(read_scalar(h->scratch.get() + SC_NORM, s));
}

// per-graph sum, sum |.|, sum of squares of a level-1 vector (map: natural -> stored index)
static void graph_stats(lamg_ctx *h, const double *v, const int32_t *map, cudaStream_t s, std::vector<double> &out) {
    const int32_t G = h->ngraphs;
    k_graph_stats<<<std::min(G, 4096), 1024, 0, s>>>(G, h->gptr_d.get(), map, v, h->gstat.get());
    LAMG_CHECK_LAUNCH();
    out.resize(3 * (size_t)G);
    LAMG_CUDA(cudaMemcpyAsync(out.data(), h->gstat.get(), sizeof(double) * 3 * G, cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
}

// out may be g (in place): each element is read and written by one thread
__global__ void k_center_graphs(int32_t n, const double *g, double *out,
                                const int32_t *__restrict__ gid, const int64_t *__restrict__ gptr,
                                const double *__restrict__ sums) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int32_t k = gid[i];
        out[i] = g[i] - sums[k] / (double)(gptr[k + 1] - gptr[k]);
    }
}

__global__ void k_add_const(int32_t n, double *__restrict__ v, double c) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] += c;
}

void solve_device(lamg_ctx *h, const double *b, double *x, double tol, lamg_precision p, cudaStream_t s,
                  lamg_stats *st) {
    auto t0 = std::chrono::steady_clock::now();
    prepare(h);
    const int32_t n = h->lv[0].n;
    const SolveLevel &V0 = h->lv[0];
    double *xb = h->v64[0].x.get(), *bb = h->v64[0].b.get();
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), b, bb);
    LAMG_CHECK_LAUNCH();
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), x, xb);
    LAMG_CHECK_LAUNCH();
    const int32_t G = h->ngraphs;
    double sb, ab, bn;
    std::vector<double> gbn(G), grn(G), gst;
    if (G > 1) {
        // a union of graphs: b must be zero-sum on every graph; each graph has its own ||b_g||
        graph_stats(h, bb, h->iperm0.get(), s, gst);
        if (h->opt.project_rhs) {  // solve for b minus its mean on every graph (the device stats start with the sums)
            k_center_graphs<<<ceil_div(n, 256), 256, 0, s>>>(n, bb, bb, h->gid0.get(), h->gptr_d.get(), h->gstat.get());
            LAMG_CHECK_LAUNCH();
            graph_stats(h, bb, h->iperm0.get(), s, gst);
        }
        bn = 0.0;
        for (int32_t g = 0; g < G; g++) {
            LAMG_REQUIRE(std::fabs(gst[g]) <= 1e-10 * (gst[G + g] > 0 ? gst[G + g] : 1.0),
                         LAMG_ERR_RHS_NOT_ZERO_SUM, "right-hand side is not zero-sum on graph " + std::to_string(g));
            gbn[g] = std::sqrt(gst[2 * G + g]);
            bn += gst[2 * G + g];
        }
        bn = std::sqrt(bn);
    } else {
        rhs_norms(h, bb, s, sb, ab, bn);
        if (h->opt.project_rhs && sb != 0.0) {  // solve for b minus its mean
            k_add_const<<<ceil_div(n, 256), 256, 0, s>>>(n, bb, -sb / (double)n);
            LAMG_CHECK_LAUNCH();
            rhs_norms(h, bb, s, sb, ab, bn);
        }
        LAMG_REQUIRE(std::fabs(sb) <= 1e-10 * (ab > 0 ? ab : 1.0), LAMG_ERR_RHS_NOT_ZERO_SUM,
                     "right-hand side is not zero-sum");
    }
    const double r0 = resnorm64(h, s);
    double rn = r0;
    if (G > 1) {
        graph_stats(h, h->r64.get(), h->iperm0.get(), s, gst);
        for (int32_t g = 0; g < G; g++) grn[g] = std::sqrt(gst[2 * G + g]);
    }
    // stopping test: ||r|| <= tol ||b||, on every graph of a union
    auto pending = [&]() {
        if (G == 1) return rn > tol * bn;
        for (int32_t g = 0; g < G; g++)
            if (!(grn[g] <= tol * gbn[g])) return true;
        return false;
    };
    const int adaptive = h->opt.adaptive;
    const int kind = p == LAMG_FP64 ? 0 : 1;
    const int per_step = p == LAMG_FP64 ? 1 : std::max(1, h->opt.ir_inner);
    int steps = 0, cycles = 0;
    std::vector<double> gn2(G);
    while (pending() && cycles < h->opt.max_cycles) {
        run_step(h, kind, adaptive, s);
        LAMG_CUDA(cudaMemcpyAsync(h->host_pinned, h->scratch.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
        if (G > 1)
            LAMG_CUDA(cudaMemcpyAsync(gn2.data(), h->gnorm.get(), sizeof(double) * G, cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaStreamSynchronize(s));
        after_step(h, kind, s);
        rn = std::sqrt(*h->host_pinned);
        for (int32_t g = 0; g < G && G > 1; g++) grn[g] = std::sqrt(gn2[g]);
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
    if (G > 1) {
        L.rel_res = 0.0;
        h->grel.assign(G, 0.0);
        for (int32_t g = 0; g < G; g++) {
            h->grel[g] = gbn[g] > 0 ? grn[g] / gbn[g] : 0.0;
            L.rel_res = std::max(L.rel_res, h->grel[g]);
        }
    }
    L.acf = (cycles > 0 && r0 > 0 && rn > 0) ? std::pow(rn / r0, 1.0 / cycles) : 0.0;
    L.t_setup_s = h->t_setup_s;
    L.t_solve_s = std::chrono::duration<double>(t1 - t0).count();
    L.status = (rn == rn && !pending()) ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
    if (st) *st = L;
    LAMG_REQUIRE(rn == rn, LAMG_ERR_NOT_CONVERGED, "solve produced NaN");
    if (L.status != LAMG_OK) throw Error{LAMG_ERR_NOT_CONVERGED, "max_cycles reached before tol"};
}

void cycle_device(lamg_ctx *h, const double *b, double *x, int32_t adaptive, cudaStream_t s) {
    prepare(h);
    const int32_t n = h->lv[0].n;
    const SolveLevel &V0 = h->lv[0];
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), b, h->v64[0].b.get());
    LAMG_CHECK_LAUNCH();
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), x, h->v64[0].x.get());
    LAMG_CHECK_LAUNCH();
    run_step(h, 2, adaptive, s);
    k_scatter_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), h->v64[0].x.get(), x);
    LAMG_CHECK_LAUNCH();
    LAMG_CUDA(cudaStreamSynchronize(s));
    after_step(h, 2, s);
}

// One cycle without any allocation: the handle's buffers and program must
// exist already; the engine scratch is the library's fixed device array.
void cycle_device_noalloc(lamg_ctx *h, const double *b, double *x, int32_t adaptive, cudaStream_t s) {
    LAMG_REQUIRE(!h->v64.empty() && h->scratch.get() && h->r64.get() && engine_noalloc_ready(h, adaptive),
                 LAMG_ERR_ARG,
                 "lamg_cycle_noalloc: handle not prepared (call lamg_cycle once with the same adaptive flag)");
    const int32_t n = h->lv[0].n;
    const SolveLevel &V0 = h->lv[0];
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), b, h->v64[0].b.get());
    LAMG_CHECK_LAUNCH();
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), x, h->v64[0].x.get());
    LAMG_CHECK_LAUNCH();
    int32_t *err = engine_run_noalloc(h, adaptive, adaptive ? h->opt.mu_adaptive : h->opt.mu_flat, s);
    k_scatter_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), h->v64[0].x.get(), x);
    LAMG_CHECK_LAUNCH();
    int32_t e = 0;
    LAMG_CUDA(cudaMemcpyAsync(&e, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    LAMG_REQUIRE(e == 0, LAMG_ERR_TIMEOUT, "cycle engine: grid barrier timed out");
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
    prepare(h);
    const int32_t n = h->lv[0].n;
    Tmp<double> gz(n, s);
    double *out = h->scratch.get() + SC_NORM + 8;
    if (h->ngraphs > 1) {
        // project g to zero mean on every graph of the union
        std::vector<double> gst;
        graph_stats(h, g, nullptr, s, gst);
        k_center_graphs<<<ceil_div(n, 256), 256, 0, s>>>(n, g, gz.get(), h->gidnat.get(), h->gptr_d.get(),
                                                         h->gstat.get());
        LAMG_CHECK_LAUNCH();
    } else {
        reduce_to(g, n, 0, h->scratch.get() + SC_PART, out, s);
        k_center<<<ceil_div(n, 256), 256, 0, s>>>(n, g, gz.get(), out);
        LAMG_CHECK_LAUNCH();
    }
    LAMG_CUDA(cudaMemsetAsync(lambda, 0, sizeof(double) * n, s));
    solve_device(h, gz.get(), lambda, tol, p, s, st);
    if (dw && m > 0) {
        k_edge_grad<<<ceil_div(m, 256), 256, 0, s>>>(m, eu, ev, lambda, x, dw, dw32);
        LAMG_CHECK_LAUNCH();
    }
    LAMG_CUDA(cudaStreamSynchronize(s));
}

void release_solve(lamg_ctx *h) {
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    h->prof_ev.clear();
    if (h->host_pinned) cudaFreeHost(h->host_pinned);
    h->host_pinned = nullptr;
}

}  // namespace lamg
