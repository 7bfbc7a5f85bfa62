// api.cu -- the extern "C" entry points declared in include/lamg.h.  Each one
// validates its arguments, runs the device work on the caller's stream and
// converts every failure into a lamg_status (never aborts).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "lamg_internal.cuh"

namespace lamg {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void set_last_error(const std::string &msg) { g_last_error = msg; }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }

template <class F>
static lamg_status guarded(F &&f) {
    try {
        f();
        g_last_error.clear();
        return LAMG_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return LAMG_ERR_OOM;
    } catch (...) {
        g_last_error = "unknown error";
        return LAMG_ERR_CUDA;
    }
}


// Two-level steps per level in one cycle, by replaying the schedule of the
// cycle (the k-th coarse correction of level l runs ceil((k+1) g) - ceil(k g)
// steps of level l+1, counters reset per cycle).
static void count_steps(lamg_ctx *h, int l, int theta, std::vector<int32_t> &visits,
                        std::vector<double> &steps) {
    for (int i = 0; i < theta; i++) {
        steps[l] += 1.0;
        if (l + 1 < h->L - 1) {
            const int32_t k = visits[l]++;
            const double g = h->sl[l].gamma_l;
            int th = (int)(std::ceil((double)(k + 1) * g) - std::ceil((double)k * g));
            th = th < 1 ? 1 : (th > 2 ? 2 : th);
            count_steps(h, l + 1, th, visits, steps);
        } else {
            steps[l + 1] += 1.0;  // one coarsest solve per step of level L-2
        }
    }
}

// Algorithmic bytes of one cycle: per two-level step at level l, (nu1 + nu2)
// sweeps, a residual (sweep bytes + r write), restriction (r read + member
// index + b^c, x^c writes), the prolongation (agg + x read/write + x^c
// gather); plus the coarsest solves (dense inverse read, or its sweeps).
// Algorithmic bytes of one cycle with `cols` right-hand sides: matrix bytes once,
// vector bytes once per column (the batched engine reads each entry once for all
// the columns of a run).
int64_t cycle_bytes(lamg_ctx *h, int wb, int cols) {
    const int L = h->L;
    auto level_bytes = [&](const SolveLevel &V) {
        return (double)V.nnz * (4 + wb) + (double)(V.n + 1) * 4 + (double)cols * V.n * wb * 3;
    };
    auto coarse_bytes = [&](const SolveLevel &C) {
        return C.dense ? (double)C.n * C.n * 8 + (double)cols * C.n * 16 : h->opt.coarse_sweeps * level_bytes(C);
    };
    if (L == 1) return (int64_t)coarse_bytes(h->lv[0]);
    std::vector<int32_t> visits(L, 0);
    std::vector<double> steps(L, 0.0);
    count_steps(h, 0, 1, visits, steps);
    double total = 0.0;
    for (int l = 0; l + 1 < L; l++) {
        const SolveLevel &V = h->lv[l];
        const double sw = level_bytes(V);
        const double res = sw + (double)cols * V.n * wb;
        const double rst = (double)V.n * 4 + (double)cols * ((double)V.n * wb + (double)h->lv[l + 1].n * 2 * wb);
        const double pro = (double)V.n * 4 + (double)cols * V.n * 2 * wb;
        if (V.elim) {   // no sweeps; restriction and back-substitution are one CSR pass together
            total += steps[l] * (res + sw + (double)cols * h->lv[l + 1].n * 2 * wb + pro);
            continue;
        }
        total += steps[l] * ((h->opt.nu1 + h->opt.nu2) * sw + res + rst + pro);
    }
    total += steps[L - 1] * coarse_bytes(h->lv[L - 1]);
    return (int64_t)total;
}

}  // namespace lamg

using namespace lamg;

extern "C" {

void lamg_default_options(lamg_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->struct_size = (int32_t)sizeof(lamg_options);
    o->gamma = 1.5;
    o->k_finest = 4;
    o->k_max = 10;
    o->k_step = 1;
    o->nu_tv = 3;
    o->nu1 = 1;
    o->nu2 = 2;
    o->n_coarsest = 150;
    o->q_max = 2.5;
    o->hub_factor = 8.0;
    o->weak_tol = 1e-8;
    o->alpha_stall = 0.95;
    o->relax_fast_ratio = 0.0;
    o->max_rounds = 8;
    o->max_levels = 100;
    o->dense_max = 1024;
    o->coarse_sweeps = 5;
    o->mu_flat = 4.0 / 3.0;
    o->seed = 1;
    o->adaptive = 1;
    o->max_cycles = 200;
    o->ir_inner = 2;
    o->validate = 1;
    o->keep_setup_data = 0;
    o->project_rhs = 0;
    o->mu_adaptive = 1.0;
    o->gamma_coarse_max = 2.0;
    o->elim = 0;
    o->elim_min_frac = 0.1;
    o->lgmg_nx = 0;
    o->agg_rule = 2;
    o->recomb_finest = 1;
    o->relax_rule = 0;
    o->colour_rule = 0;
    o->negative_weights = 0;
}

const char *lamg_last_error(void) { return g_last_error.c_str(); }

static lamg_status setup_impl(int32_t ngraphs, const int64_t *graph_ptr, int64_t n, const int64_t *row_ptr,
                              const int32_t *col, const void *w, int32_t w_is_fp32, const lamg_options *opt,
                              lamg_stream stream, lamg_handle *out) {
    if (out) *out = nullptr;
    lamg_ctx *h = nullptr;
    lamg_status st = guarded([&] {
        LAMG_REQUIRE(out != nullptr, LAMG_ERR_ARG, "out is NULL");
        LAMG_REQUIRE(n >= 1 && n < ((int64_t)1 << 31), LAMG_ERR_ARG, "n must be in [1, 2^31)");
        LAMG_REQUIRE(row_ptr != nullptr, LAMG_ERR_ARG, "NULL row_ptr");
        LAMG_REQUIRE(ngraphs >= 1 && graph_ptr != nullptr, LAMG_ERR_ARG, "num_graphs must be >= 1 with graph_ptr");
        LAMG_REQUIRE(graph_ptr[0] == 0 && graph_ptr[ngraphs] == n, LAMG_ERR_ARG,
                     "graph_ptr must start at 0 and end at n");
        for (int32_t g = 0; g < ngraphs; g++)
            LAMG_REQUIRE(graph_ptr[g + 1] > graph_ptr[g], LAMG_ERR_ARG, "graph_ptr must be strictly increasing");
        // the options are checked before anything is allocated
        lamg_options o;
        if (opt) o = *opt; else lamg_default_options(&o);
        LAMG_REQUIRE(o.struct_size == (int32_t)sizeof(lamg_options), LAMG_ERR_ARG,
                     "lamg_options.struct_size does not match this library (fill it with lamg_default_options)");
        LAMG_REQUIRE(o.gamma >= 1.0 && o.nu_tv >= 0 && o.nu1 >= 0 && o.nu2 >= 0 && o.k_finest >= 1 &&
                         o.max_rounds >= 1 && o.max_levels >= 1 && o.dense_max >= 1 &&
                         o.gamma_coarse_max >= 1.0 && o.gamma_coarse_max <= 2.0 &&
                         o.mu_adaptive > 0.0 && o.mu_adaptive < 4.0 && o.mu_flat > 0.0 && o.mu_flat < 4.0 &&
                         o.q_max > 0.0 && o.n_coarsest >= 1 && o.coarse_sweeps >= 0 &&
                         o.agg_rule >= 0 && o.agg_rule <= 2 && (o.recomb_finest == 0 || o.recomb_finest == 1) &&
                         (o.relax_rule == 0 || o.relax_rule == 1) && o.sb_work32 >= 0 && o.sb_work64 >= 0 &&
                         o.tail_work32 >= 0 && o.tail_work64 >= 0 && (o.colour_rule == 0 || o.colour_rule == 1) &&
                         (o.negative_weights == 0 || o.negative_weights == 1),
                     LAMG_ERR_ARG, "invalid options");
        auto t0 = std::chrono::steady_clock::now();
        h = new lamg_ctx();
        h->ngraphs = ngraphs;
        h->gptr.assign(graph_ptr, graph_ptr + ngraphs + 1);
        h->opt = o;
        cudaStream_t s = (cudaStream_t)stream;
        if (h->opt.validate)
            validate_graph(n, row_ptr, col, w, w_is_fp32, s, ngraphs, graph_ptr, h->opt.negative_weights);
        build_hierarchy(h, n, row_ptr, col, w, w_is_fp32, s);
        build_solve_layout(h, s);
        h->n = n;
        if (ngraphs > 1) build_graph_maps(h, s);
        auto t1 = std::chrono::steady_clock::now();
        h->t_setup_s = std::chrono::duration<double>(t1 - t0).count();
        int64_t tot = 0;
        for (auto &V : h->lv) tot += V.nnz;
        h->last.levels = h->L;
        h->last.t_setup_s = h->t_setup_s;
        h->last.nnz_total = tot;
        h->last.bytes_per_cycle = cycle_bytes(h, 8, 1);
        h->last.bytes_per_cycle32 = cycle_bytes(h, 4, 1);
    });
    if (st != LAMG_OK) {
        if (h) { release_solve(h); delete h; }
        return st;
    }
    *out = h;
    return LAMG_OK;
}

lamg_status lamg_setup(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                       int32_t w_is_fp32, const lamg_options *opt, lamg_stream stream, lamg_handle *out) {
    const int64_t gp[2] = {0, n};
    return setup_impl(1, gp, n, row_ptr, col, w, w_is_fp32, opt, stream, out);
}

lamg_status lamg_setup_graphs(int32_t num_graphs, const int64_t *graph_ptr, int64_t n, const int64_t *row_ptr,
                              const int32_t *col, const void *w, int32_t w_is_fp32, const lamg_options *opt,
                              lamg_stream stream, lamg_handle *out) {
    if (out) *out = nullptr;
    if (num_graphs < 1 || !graph_ptr) {
        set_last_error("num_graphs must be >= 1 with graph_ptr");
        return LAMG_ERR_ARG;
    }
    return setup_impl(num_graphs, graph_ptr, n, row_ptr, col, w, w_is_fp32, opt, stream, out);
}

lamg_status lamg_solve(lamg_handle h, const double *b, double *x, double tol, lamg_precision p,
                       lamg_stream stream, lamg_stats *st) {
    return guarded([&] {
        LAMG_REQUIRE(h && b && x, LAMG_ERR_ARG, "NULL argument");
        LAMG_REQUIRE(p == LAMG_FP64 || p == LAMG_FP32_IR, LAMG_ERR_ARG, "unknown precision");
        LAMG_REQUIRE(tol >= 0.0, LAMG_ERR_ARG, "tol must be >= 0");
        solve_device(h, b, x, tol, p, (cudaStream_t)stream, st);
    });
}

lamg_status lamg_solve_host(lamg_handle h, const double *b_host, double *x_host, double tol,
                            lamg_precision p, lamg_stream stream, lamg_stats *st) {
    return guarded([&] {
        LAMG_REQUIRE(h && b_host && x_host, LAMG_ERR_ARG, "NULL argument");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t bytes = sizeof(double) * (size_t)h->n;
        if (!h->bnat.get()) { h->bnat.alloc(h->n); h->xnat.alloc(h->n); }
        LAMG_CUDA(cudaMemcpyAsync(h->bnat.get(), b_host, bytes, cudaMemcpyHostToDevice, s));
        LAMG_CUDA(cudaMemcpyAsync(h->xnat.get(), x_host, bytes, cudaMemcpyHostToDevice, s));
        lamg_status inner = LAMG_OK;
        try {
            solve_device(h, h->bnat.get(), h->xnat.get(), tol, p, s, st);
        } catch (const Error &e) {
            if (e.status != LAMG_ERR_NOT_CONVERGED) throw;
            inner = e.status;
        }
        LAMG_CUDA(cudaMemcpyAsync(x_host, h->xnat.get(), bytes, cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaStreamSynchronize(s));
        if (inner != LAMG_OK) throw Error{inner, "max_cycles reached before tol"};
    });
}

lamg_status lamg_solve_batched(lamg_handle h, int32_t nrhs, const double *B, double *X, int64_t ld,
                               double tol, lamg_precision p, lamg_stream stream, lamg_stats *st) {
    return guarded([&] {
        LAMG_REQUIRE(h && B && X && nrhs >= 1 && ld >= nrhs, LAMG_ERR_ARG, "bad batched arguments");
        solve_batched_device(h, nrhs, B, X, ld, tol, p, (cudaStream_t)stream, st);
    });
}

lamg_status lamg_autotune_batched(lamg_handle h, int32_t nrhs, lamg_precision precision, lamg_stream stream,
                                  int32_t *chosen_cols, double *ms_host) {
    return guarded([&] {
        LAMG_REQUIRE(h && nrhs >= 1, LAMG_ERR_ARG, "bad autotune arguments");
        autotune_batched(h, nrhs, precision, (cudaStream_t)stream, chosen_cols, ms_host);
    });
}

lamg_status lamg_set_batch_cols(lamg_handle h, int32_t cols) {
    return guarded([&] {
        LAMG_REQUIRE(h, LAMG_ERR_ARG, "NULL handle");
        set_batch_cols(h, cols);
    });
}

lamg_status lamg_adjoint(lamg_handle h, const double *x, const double *g, double *lambda,
                         const int32_t *eu, const int32_t *ev, int64_t m, void *dw, int32_t dw_is_fp32,
                         double tol, lamg_precision p, lamg_stream stream, lamg_stats *st) {
    return guarded([&] {
        LAMG_REQUIRE(h && x && g && lambda, LAMG_ERR_ARG, "NULL argument");
        LAMG_REQUIRE(!dw || (eu && ev && m >= 0), LAMG_ERR_ARG, "edge arrays required for dw");
        adjoint_device(h, x, g, lambda, eu, ev, m, dw, dw_is_fp32, tol, p, (cudaStream_t)stream, st);
    });
}

void lamg_free(lamg_handle h) {
    if (!h) return;
    cudaDeviceSynchronize();
    release_solve(h);
    delete h;
}

lamg_status lamg_level_info(lamg_handle h, int32_t level, int64_t *info) {
    return guarded([&] {
        LAMG_REQUIRE(h && info && level >= 0 && level < h->L, LAMG_ERR_ARG, "bad level");
        const SetupLevel &S = h->sl[level];
        std::memset(info, 0, sizeof(int64_t) * 16);
        info[0] = S.n; info[1] = S.nnz; info[2] = S.ncolours; info[3] = S.K; info[4] = S.nc;
        info[5] = S.rounds; info[6] = S.sel_round; info[7] = S.coarsest; info[8] = S.stop_reason;
        std::memcpy(&info[9], &S.alpha, 8);
        std::memcpy(&info[10], &S.gamma_l, 8);
        std::memcpy(&info[11], &S.tv_ratio, 8);
        info[12] = S.jp_rounds;
        info[13] = h->lv.empty() ? 0 : h->lv[level].dense;
        info[14] = S.elim;
        info[15] = S.nF;
    });
}

lamg_status lamg_level_copy(lamg_handle h, int32_t level, int32_t field, void *dst, int64_t bytes) {
    return guarded([&] {
        LAMG_REQUIRE(h && dst && level >= 0 && level < h->L, LAMG_ERR_ARG, "bad level");
        const SetupLevel &S = h->sl[level];
        const void *src = nullptr;
        size_t need = 0;
        std::vector<int64_t> rp64;
        switch (field) {
            case 0: {
                std::vector<int32_t> rp32(S.n + 1);
                LAMG_CUDA(cudaMemcpy(rp32.data(), S.rp.get(), sizeof(int32_t) * (S.n + 1), cudaMemcpyDeviceToHost));
                rp64.assign(rp32.begin(), rp32.end());
                need = sizeof(int64_t) * (S.n + 1);
                LAMG_REQUIRE(bytes == (int64_t)need, LAMG_ERR_ARG, "size mismatch");
                std::memcpy(dst, rp64.data(), need);
                return;
            }
            case 1: src = S.col.get(); need = S.col.bytes(); break;
            case 2: src = S.w.get(); need = S.w.bytes(); break;
            case 3: src = S.colour.get(); need = S.colour.bytes(); break;
            case 4: src = S.agg.get(); need = S.agg.bytes(); break;
            case 5: src = S.state.get(); need = S.state.bytes(); break;
            case 6: src = S.hub.get(); need = S.hub.bytes(); break;
            case 7: src = S.tv.get(); need = S.tv.bytes(); break;
            case 8: src = S.aff.get(); need = S.aff.bytes(); break;
            case 9: src = S.q.get(); need = S.q.bytes(); break;
            case 10: src = S.score.get(); need = S.score.bytes(); break;
            case 11: src = S.cidx.get(); need = S.cidx.bytes(); break;
            default: break;
        }
        const bool empty_ok = (field == 1 || field == 2) && S.nnz == 0;
        LAMG_REQUIRE(src != nullptr || empty_ok, LAMG_ERR_ARG, "field not available on this level");
        LAMG_REQUIRE(bytes == (int64_t)need, LAMG_ERR_ARG, "size mismatch");
        if (need) LAMG_CUDA(cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost));
    });
}

lamg_status lamg_cycle(lamg_handle h, const double *b, double *x, int32_t adaptive, lamg_stream stream) {
    return guarded([&] {
        LAMG_REQUIRE(h && b && x, LAMG_ERR_ARG, "NULL argument");
        cycle_device(h, b, x, adaptive, (cudaStream_t)stream);
    });
}

lamg_status lamg_cycle_noalloc(lamg_handle h, const double *b, double *x, int32_t adaptive, lamg_stream stream) {
    return guarded([&] {
        LAMG_REQUIRE(h && b && x, LAMG_ERR_ARG, "NULL argument");
        cycle_device_noalloc(h, b, x, adaptive, (cudaStream_t)stream);
    });
}

lamg_status lamg_graph_residuals(lamg_handle h, double *rel_res_host) {
    return guarded([&] {
        LAMG_REQUIRE(h && rel_res_host, LAMG_ERR_ARG, "NULL argument");
        LAMG_REQUIRE(h->ngraphs > 1, LAMG_ERR_ARG, "the handle holds one graph (use lamg_stats.rel_res)");
        LAMG_REQUIRE((int32_t)h->grel.size() == h->ngraphs, LAMG_ERR_ARG, "no solve has run on this handle");
        std::memcpy(rel_res_host, h->grel.data(), sizeof(double) * h->ngraphs);
    });
}

lamg_status lamg_barrier_selftest(int32_t hold_one_block, lamg_stream stream) {
    return guarded([&] {
        const int32_t e = barrier_selftest(hold_one_block, (cudaStream_t)stream);
        LAMG_REQUIRE(e == 0, LAMG_ERR_TIMEOUT, "grid barrier: wait ran out (a block never arrived)");
    });
}

lamg_status lamg_profile(lamg_handle h, int32_t enable, double *avg_ms, int64_t *count, int64_t *bytes) {
    return guarded([&] {
        LAMG_REQUIRE(h, LAMG_ERR_ARG, "NULL handle");
        if (avg_ms) *avg_ms = h->prof_count ? h->prof_ms / (double)h->prof_count : 0.0;
        if (count) *count = h->prof_count;
        if (bytes) *bytes = h->prof_bytes;
        if (enable) { h->prof_ms = 0.0; h->prof_count = 0; }
        h->prof_on = enable ? 1 : 0;
    });
}

lamg_status lamg_op_times(lamg_handle h, int32_t mode, int32_t cap, int32_t *level, int32_t *op,
                          int32_t *single_block, int64_t *count, double *total_ns, int32_t *n_rows) {
    return guarded([&] {
        LAMG_REQUIRE(h, LAMG_ERR_ARG, "NULL handle");
        LAMG_REQUIRE(mode >= -1 && mode <= 1, LAMG_ERR_ARG, "mode must be -1, 0 or 1");
        std::vector<unsigned long long> t;
        engine_op_times(h, mode, t);
        if (mode != 0) return;
        LAMG_REQUIRE(cap == 0 || (level && op && single_block && count && total_ns), LAMG_ERR_ARG,
                     "NULL output array");
        int32_t rows = 0;
        for (int l = 0; l < 128; l++)
            for (int ty = 0; ty < 32; ty++)
                for (int sb = 0; sb < 2; sb++) {
                    const int key = (l * 32 + ty) * 2 + sb;
                    if (!t[2 * key + 1]) continue;
                    if (rows < cap) {
                        level[rows] = l;
                        op[rows] = ty;
                        single_block[rows] = sb;
                        count[rows] = (int64_t)t[2 * key + 1];
                        total_ns[rows] = (double)t[2 * key];
                    }
                    rows++;
                }
        if (n_rows) *n_rows = rows;
    });
}

lamg_status lamg_launch_count(int64_t *count) {
    return guarded([&] {
        LAMG_REQUIRE(count, LAMG_ERR_ARG, "NULL argument");
        *count = launch_count();
    });
}

}  // extern "C"
