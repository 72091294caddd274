// The C ABI (include/cfc_gb300.h): argument checks, error translation,
// hierarchy handles, and the launch counters / event timers.
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

namespace cfc {

namespace {
thread_local std::string t_last_error;

// ---------------------------------------------------------------- stats
std::atomic<uint64_t> g_launches_total{0};
std::atomic<uint64_t> g_launches[LAP_KF_COUNT];
std::atomic<int> g_timing{0};
std::atomic<int> g_log_on{0};
std::mutex g_log_mu;
std::vector<int32_t> g_log;

struct Pending {
    int family;
    double bytes;
    cudaEvent_t a, b;
};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;
double g_ms[LAP_KF_COUNT];
double g_bytes[LAP_KF_COUNT];

cudaEvent_t get_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    CFC_CUDA(cudaEventCreate(&e));
    return e;
}

// folds completed timings into the totals (caller holds g_mu)
void drain_locked() {
    for (auto &p : g_pending) {
        float ms = 0.f;
        CFC_CUDA(cudaEventSynchronize(p.b));
        CFC_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        g_ms[p.family] += ms;
        g_bytes[p.family] += p.bytes;
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
}
}  // namespace

void set_last_error(const std::string &s) { t_last_error = s; }
void clear_last_error() { t_last_error.clear(); }

bool stats_detailed() {
    return g_timing.load(std::memory_order_relaxed) != 0 || g_log_on.load(std::memory_order_relaxed) != 0;
}
void stats_launches(int64_t out[LAP_KF_COUNT]) {
    for (int f = 0; f < LAP_KF_COUNT; ++f) out[f] = (int64_t)g_launches[f].load(std::memory_order_relaxed);
}
void stats_add_launches(const int64_t delta[LAP_KF_COUNT], int64_t times) {
    for (int f = 0; f < LAP_KF_COUNT; ++f) {
        const int64_t d = delta[f] * times;
        g_launches[f].fetch_add((uint64_t)d, std::memory_order_relaxed);
        g_launches_total.fetch_add((uint64_t)d, std::memory_order_relaxed);
    }
}

LaunchScope::LaunchScope(int fam, cudaStream_t s, double algorithmic_bytes)
    : family(fam), stream(s), bytes(algorithmic_bytes) {
    g_launches_total.fetch_add(1, std::memory_order_relaxed);
    g_launches[fam].fetch_add(1, std::memory_order_relaxed);
    if (g_log_on.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_log_mu);
        g_log.push_back(fam);
    }
    if (g_timing.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_pending.size() > 65536) drain_locked();
        start = get_event();
        if (cudaEventRecord(start, s) != cudaSuccess) {
            cudaGetLastError();
            g_free_events.push_back(start);
            start = nullptr;
        }
    }
}

LaunchScope::~LaunchScope() {
    if (!start) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t stop = nullptr;
    if (!g_free_events.empty()) {
        stop = g_free_events.back();
        g_free_events.pop_back();
    } else if (cudaEventCreate(&stop) != cudaSuccess) {
        cudaGetLastError();
        g_free_events.push_back(start);
        return;
    }
    if (cudaEventRecord(stop, stream) != cudaSuccess) {
        cudaGetLastError();
        g_free_events.push_back(start);
        g_free_events.push_back(stop);
        return;
    }
    g_pending.push_back(Pending{family, bytes, start, stop});
}

cudaMemPool_t library_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    CFC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        CFC_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t thr = ~uint64_t(0);
        CFC_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
        pools[dev] = p;
    }
    return pools[dev];
}

bool is_device_pointer(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

const void *mapped_host_pointer(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

LevelView view(const Level &L) {
    LevelView v;
    v.n = L.n;
    v.rowptr = L.rowptr.get();
    v.col = L.col.get();
    v.w32 = L.w32.get();
    v.deg32 = L.deg32.get();
    v.dinv32 = L.dinv32.get();
    v.wbf = nullptr;
    v.w64 = L.w64.get();
    v.deg64 = L.deg64.get();
    v.dinv64 = L.dinv64.get();
    v.n_chunks = L.n_chunks;
    v.n_long = L.n_long;
    v.long_row = L.long_row;
    v.chunk = L.chunk;
    v.chunk_row = L.chunk_row.get();
    v.chunk_begin = L.chunk_begin.get();
    v.chunk_long = L.chunk_long.get();
    v.long_first = L.long_first.get();
    v.long_of_row = L.long_of_row.get();
    v.order = L.order.get();
    v.chunk_order = L.chunk_order.get();
    v.long_count = nullptr;  // set by the solve that launches on the level
    return v;
}

LevelView view_bf16(const Level &L) {
    LevelView v = view(L);
    v.wbf = L.wbf.get();
    v.deg32 = L.degbf.get();
    v.dinv32 = L.dinvbf.get();
    return v;
}

LevelView pull_view(const Level &E) {
    LevelView v{};
    v.n = E.pull_ptr.get() ? (int32_t)(E.pull_ptr.n - 1) : 0;
    v.rowptr = E.pull_ptr.get();
    v.col = E.pull_u.get();
    v.w32 = E.pull_c32.get();
    v.w64 = E.pull_c64.get();
    v.n_chunks = E.pull_n_chunks;
    v.n_long = E.pull_n_long;
    v.long_row = E.pull_long_row;
    v.chunk = E.pull_chunk;
    v.chunk_row = E.pull_chunk_row.get();
    v.chunk_begin = E.pull_chunk_begin.get();
    v.chunk_long = E.pull_chunk_long.get();
    v.long_first = E.pull_long_first.get();
    v.long_of_row = E.pull_long_of_row.get();
    return v;  // natural row and chunk order; no degrees (the restriction reads none)
}

void release_workspace(lap_hierarchy *h, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(h->ws_mu);
    h->ws.erase(s);  // DBuf frees on the stream it was taken on
}

int64_t hierarchy_bytes(const lap_hierarchy *h) {
    auto b = [](const auto &d) { return (int64_t)(d.n * sizeof(*d.p)); };
    int64_t t = b(h->eid) + b(h->coarse_inv) + b(h->coarse_inv32);
    for (const Level &L : h->lv)
        t += b(L.rowptr) + b(L.col) + b(L.w64) + b(L.deg64) + b(L.dinv64) + b(L.w32) + b(L.deg32) + b(L.dinv32) +
             b(L.wbf) + b(L.degbf) + b(L.dinvbf) + b(L.chunk_row) + b(L.chunk_begin) + b(L.chunk_long) +
             b(L.long_first) + b(L.long_of_row) + b(L.order) + b(L.chunk_order) + b(L.agg) + b(L.mem_ptr) +
             b(L.mem) +
             b(L.keep_id) + b(L.keep_node) + b(L.e_node) + b(L.e_nb) + b(L.e_c64) + b(L.e_c32) +
             b(L.e_dinv64) + b(L.e_dinv32) + b(L.pull_ptr) + b(L.pull_e) + b(L.pull_u) + b(L.pull_c64) +
             b(L.pull_c32) + b(L.pull_chunk_row) + b(L.pull_chunk_begin) + b(L.pull_chunk_long) +
             b(L.pull_long_first) + b(L.pull_long_of_row) + b(L.jl_chunk_row) + b(L.jl_chunk_begin) +
             b(L.jl_long_first);
    return t;
}


}  // namespace cfc

using namespace cfc;

extern "C" {

void lap_default_hier_opts(lap_hier_opts_t *o) {
    if (!o) return;
    o->coarse_max = 0;  // automatic
    o->max_levels = 24;
    o->agg_passes = 2;
    o->match_rounds = 4;
    o->eager = 0;
    o->eliminate = 1;
    o->reorder = 0;
    o->aggregation = LAP_AGG_STRENGTH;
    o->hub_factor = 0;
    o->chunking = 0;
}

void lap_default_solve_opts(lap_solve_opts_t *o) {
    if (!o) return;
    o->precision = LAP_FP32_REFINED;
    o->tol = 1e-8;
    o->max_outer = 8;
    o->max_inner = 200;
    o->inner_tol = 1e-4;
    o->k_tile = 0;
    o->smoother = LAP_SMOOTH_CHEBYSHEV;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->check_every = 4;
    o->levels_used = 0;
    o->nu_coarse = 0;
    o->cycle = 0;
    o->w_levels = 0;
    o->graphs = 1;
    o->first_residual_ff = 1;
    o->coarse_scale = 0.0;
}

const char *lap_status_string(lap_status_t s) {
    switch (s) {
        case LAP_OK: return "LAP_OK";
        case LAP_EINVAL: return "LAP_EINVAL: invalid argument";
        case LAP_ENOTCONN: return "LAP_ENOTCONN: graph is not connected";
        case LAP_ENOMEM: return "LAP_ENOMEM: out of memory";
        case LAP_ENOCONV: return "LAP_ENOCONV: iteration cap reached before the tolerance";
        case LAP_ECUDA: return "LAP_ECUDA: CUDA error";
        case LAP_EBUDGET: return "LAP_EBUDGET: request exceeds a documented maximum";
        case LAP_ENOTIMPL: return "LAP_ENOTIMPL: not implemented";
        case LAP_EPENDING: return "LAP_EPENDING: request not finished";
    }
    return "unknown status";
}

const char *lap_last_error(void) { return t_last_error.c_str(); }

lap_status_t lap_build_hierarchy(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const double *w,
                                 const lap_hier_opts_t *opts, void *stream, lap_hierarchy_t **out) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(out, LAP_EINVAL, "out must not be NULL");
        *out = nullptr;
        lap_hier_opts_t o;
        lap_default_hier_opts(&o);
        if (opts) o = *opts;
        CFC_REQUIRE(o.coarse_max >= 0, LAP_EINVAL, "coarse_max must be >= 0 (0: automatic)");
        CFC_REQUIRE(o.agg_passes >= 1 && o.agg_passes <= 4, LAP_EINVAL, "agg_passes must be 1..4");
        CFC_REQUIRE(o.eliminate == 0 || o.eliminate == 1, LAP_EINVAL, "eliminate must be 0 or 1");
        CFC_REQUIRE(o.reorder >= 0 && o.reorder <= 2, LAP_EINVAL, "reorder must be 0, 1 or 2");
        CFC_REQUIRE(o.aggregation == LAP_AGG_STRENGTH || o.aggregation == LAP_AGG_AFFINITY, LAP_EINVAL,
                    "aggregation must be LAP_AGG_STRENGTH or LAP_AGG_AFFINITY");
        CFC_REQUIRE(o.hub_factor >= 0 && o.hub_factor <= 1000000, LAP_EINVAL, "hub_factor must be in [0, 1e6]");
        CFC_REQUIRE(o.chunking >= 0 && o.chunking <= 2, LAP_EINVAL, "chunking must be 0, 1 or 2");
        cudaStream_t s = (cudaStream_t)stream;
        auto *h = new lap_hierarchy();
        try {
            CFC_CUDA(cudaGetDevice(&h->device));
            cudaEvent_t e0, e1;
            CFC_CUDA(cudaEventCreate(&e0));
            CFC_CUDA(cudaEventCreate(&e1));
            CFC_CUDA(cudaEventRecord(e0, s));
            Csr64 g;
            ingest(n, m, src, dst, w, s, g);
            h->n = g.n;
            h->m = g.m;
            h->eid = std::move(g.eid);
            init_levels(*h, g, o, s);
            if (o.eager) grow_levels(*h, 0, s);
            noalloc_prepare();  // the allocation-free entry point's scratch, on this device
            CFC_CUDA(cudaEventRecord(e1, s));
            CFC_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            CFC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            h->setup_ms = ms;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            CFC_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            cudaStreamSynchronize(s);
            delete h;
            throw;
        }
        *out = h;
        return LAP_OK;
    });
}

void lap_hierarchy_destroy(lap_hierarchy_t *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    delete h;
}

lap_status_t lap_hierarchy_info(const lap_hierarchy_t *h, lap_hier_info_t *info) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(h && info, LAP_EINVAL, "NULL argument");
        std::shared_lock<std::shared_mutex> lk(h->mu);
        std::memset(info, 0, sizeof(*info));
        info->n = h->n;
        info->m = h->m;
        info->levels = (int32_t)h->lv.size();
        info->coarse_n = h->coarse_n;
        for (size_t l = 0; l < h->lv.size() && l < 32; ++l) {
            info->level_n[l] = h->lv[l].n;
            info->level_nnz[l] = h->lv[l].nnz;
        }
        info->setup_ms = h->setup_ms;
        info->weight_exp = h->wexp;
        info->fingerprint = h->fingerprint;
        info->elim_levels = h->p0;
        for (size_t l = 0; l < h->lv.size() && l < 32; ++l) info->level_row_order[l] = h->lv[l].order.get() ? 1 : 0;
        return LAP_OK;
    });
}

static lap_solve_opts_t resolve_opts(const lap_solve_opts_t *o) {
    lap_solve_opts_t r;
    lap_default_solve_opts(&r);
    if (o) r = *o;
    return r;
}

lap_status_t lap_solve_multi(lap_hierarchy_t *h, int32_t k, const double *B, double *X, const lap_solve_opts_t *o,
                             void *stream, lap_solve_info_t *info) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(h, LAP_EINVAL, "NULL hierarchy");
        return solve_multi(h, k, B, X, resolve_opts(o), (cudaStream_t)stream, info);
    });
}

lap_status_t cfc_jl_rhs(lap_hierarchy_t *h, int32_t k, uint64_t seed, double *Y, void *stream) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(h && Y, LAP_EINVAL, "NULL argument");
        CFC_REQUIRE(k >= 1 && k <= 4096, LAP_EINVAL, "need 1 <= k <= 4096");
        CFC_REQUIRE(is_device_pointer(Y), LAP_EINVAL, "Y must be a device pointer");
        jl_rhs(h, k, 0, k, k, seed, Y, (cudaStream_t)stream);
        return LAP_OK;
    });
}

lap_status_t cfc_farness_jl_rows(lap_hierarchy_t *h, int32_t k_total, int32_t row_begin, int32_t row_count,
                                 uint64_t seed, int32_t q, const int32_t *nodes, double *farness,
                                 const lap_solve_opts_t *o, void *stream) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(h, LAP_EINVAL, "NULL hierarchy");
        return farness_jl_rows(h, k_total, row_begin, row_count, seed, q, nodes, farness, resolve_opts(o),
                               (cudaStream_t)stream);
    });
}

lap_status_t cfc_farness_jl(lap_hierarchy_t *h, int32_t k, double eps, uint64_t seed, int32_t q,
                            const int32_t *nodes, double *farness, const lap_solve_opts_t *o, void *stream) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(h, LAP_EINVAL, "NULL hierarchy");
        return farness_jl(h, k, eps, seed, q, nodes, farness, resolve_opts(o), (cudaStream_t)stream);
    });
}

lap_status_t cfc_farness_from_solution(int64_t n, int32_t k, const double *Z, int32_t q, const int32_t *nodes,
                                       double *farness, void *stream) {
    return guard([&]() -> lap_status_t {
        return farness_from_solution(n, k, Z, q, nodes, farness, (cudaStream_t)stream);
    });
}

lap_status_t cfc_farness_from_solution_noalloc(int64_t n, int32_t k, const double *Z, int32_t q,
                                               const int32_t *nodes, double *farness, void *stream) {
    return guard([&]() -> lap_status_t {
        return farness_from_solution_noalloc(n, k, Z, q, nodes, farness, (cudaStream_t)stream);
    });
}

lap_status_t cfc_sample_pivots(lap_hierarchy_t *h, int32_t n_pivots, uint64_t seed, int32_t *pivots,
                               void *stream) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(h, LAP_EINVAL, "NULL hierarchy");
        return pivots_api(h, n_pivots, seed, pivots, (cudaStream_t)stream);
    });
}

lap_status_t cfc_farness_sampled(lap_hierarchy_t *h, int32_t n_pivots, uint64_t seed, int32_t q,
                                 const int32_t *nodes, double *farness, const lap_solve_opts_t *o, void *stream) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(h, LAP_EINVAL, "NULL hierarchy");
        return farness_sampled(h, n_pivots, seed, q, nodes, farness, resolve_opts(o), (cudaStream_t)stream);
    });
}

lap_status_t cfc_exact_small(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const double *w,
                             double *farness, double *closeness, void *stream) {
    return guard([&]() -> lap_status_t {
        return exact_small(n, m, src, dst, w, farness, closeness, (cudaStream_t)stream);
    });
}

lap_status_t lap_tune_save(const char *path) {
    return guard([&]() -> lap_status_t { return tune_save(path); });
}

lap_status_t lap_tune_load(const char *path, int64_t *added) {
    return guard([&]() -> lap_status_t { return tune_load(path, added); });
}

int64_t lap_tune_entries(void) { return tune_entries(); }

void lap_stats_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    try {
        drain_locked();
    } catch (...) {
    }
    g_launches_total.store(0);
    {
        std::lock_guard<std::mutex> lk2(g_log_mu);
        g_log.clear();
    }
    for (int f = 0; f < LAP_KF_COUNT; ++f) {
        g_launches[f].store(0);
        g_ms[f] = 0;
        g_bytes[f] = 0;
    }
}

void lap_stats_set_timing(int32_t on) { g_timing.store(on ? 1 : 0); }

void lap_stats_set_log(int32_t on) { g_log_on.store(on ? 1 : 0); }

lap_status_t lap_stats_read_log(int32_t *families, int64_t capacity, int64_t *count) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(count && (families || capacity <= 0), LAP_EINVAL, "NULL argument");
        std::lock_guard<std::mutex> lk(g_log_mu);
        *count = (int64_t)g_log.size();
        const int64_t c = std::min<int64_t>(capacity, (int64_t)g_log.size());
        for (int64_t i = 0; i < c; ++i) families[i] = g_log[i];
        return LAP_OK;
    });
}

lap_status_t lap_stats_read(lap_stats_t *out) {
    return guard([&]() -> lap_status_t {
        CFC_REQUIRE(out, LAP_EINVAL, "NULL argument");
        std::lock_guard<std::mutex> lk(g_mu);
        drain_locked();
        out->launches_total = g_launches_total.load();
        for (int f = 0; f < LAP_KF_COUNT; ++f) {
            out->launches[f] = g_launches[f].load();
            out->ms[f] = g_ms[f];
            out->bytes[f] = g_bytes[f];
        }
        return LAP_OK;
    });
}

}  // extern "C"
