// Request loop for farness queries on resident graphs, with continuous
// batching (include/cfc_gb300.h, cfc_server_*).  Each request runs the
// sampling estimator of Sec. 5.1 (pivots drawn as in Sec. 5.1 / Proposition
// 1, then n_pivots + q column solves and the reduction) on its own worker
// thread and CUDA stream; admission is first-come first-served, gated by a
// free slot and by the HBM budget.  The paper has no serving counterpart.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

using Clock = std::chrono::steady_clock;

namespace {
double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}
}  // namespace

struct cfc_server {
    cfc_server_opts_t o{};
    int device = 0;
    int64_t budget = 0;

    struct Graph {
        lap_hierarchy *h = nullptr;
        lap_solve_opts_t opts{};  // pinned configuration of its requests
        int64_t n = 0, bytes = 0;
        // resident pivot set: pivots and their solutions (n x kp, FP64)
        int32_t kp = 0;
        cfc::DBuf<int32_t> piv;
        cfc::DBuf<double> xs;
    };
    // guarded by mu for growth; entries never move (deque) or go while serving
    std::deque<Graph> graphs;

    struct Request {
        int64_t id = 0;
        int32_t graph = 0, q = 0, kk = 0;
        uint64_t seed = 0;
        std::vector<int32_t> nodes;
        std::vector<double> far;
        int64_t bytes = 0;
        Clock::time_point t_submit, t_admit, t_done;
        lap_status_t status = LAP_EPENDING;
        bool done = false;
    };

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;                          // waiting, in arrival order
    std::map<int64_t, std::unique_ptr<Request>> reqs;  // not yet polled
    int64_t next_id = 1;
    int64_t graph_bytes = 0, inflight_bytes = 0, peak_inflight_bytes = 0;
    int in_flight = 0, max_in_flight = 0, max_batch = 0;
    bool stopping = false;
    // statistics of completed requests
    std::vector<double> lat_ms;
    int64_t submitted = 0, completed = 0, rhs_done = 0;
    bool have_span = false;
    Clock::time_point span0, span1;

    std::vector<cudaStream_t> streams;  // one per slot
    cudaStream_t admin = nullptr;        // graph builds and their tuning
    std::mutex admin_mu;
    std::vector<std::thread> workers;

    // device memory of one request: its right-hand side and solution blocks
    // (FP64) and the solver workspace on its stream, at the padded width
    static int64_t request_bytes(int64_t n, int32_t cols) {
        const int64_t ld = ((cols + 63) / 64) * 64;
        return n * ld * 64 + (int64_t)(16 << 20);
    }

    bool head_admissible() const {
        if (queue.empty()) return false;
        const Request &r = *reqs.at(queue.front());
        return graph_bytes + inflight_bytes + r.bytes <= budget;
    }

    // columns a batch may hold: the option, at most 4096 columns and 64 tiles
    // of the graph's pinned tile width (so the tile, and with it every
    // column's bits, is the same as for the request alone)
    int64_t batch_limit(const Graph &g) const {
        const int64_t kt = g.opts.k_tile > 0 ? g.opts.k_tile : 64;
        return std::max<int64_t>(1, std::min<int64_t>({(int64_t)o.batch_columns, 4096, 64 * kt}));
    }

    void worker(int slot) {
        cudaSetDevice(device);
        cudaStream_t s = streams[slot];
        for (;;) {
            // the head of the queue, and (continuous batching) the queued
            // requests on the same graph and of the same kind that fit beside
            // it: one block solve for all their columns
            std::vector<Request *> batch;
            const Graph *gp = nullptr;
            int64_t batch_bytes = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stopping || head_admissible(); });
                if (stopping) return;
                Request *r = reqs.at(queue.front()).get();
                queue.pop_front();
                gp = &graphs[r->graph];
                batch.push_back(r);
                int64_t cols = r->kk + r->q;
                batch_bytes = r->bytes;
                const int64_t limit = batch_limit(*gp);
                for (auto it = queue.begin(); it != queue.end() && cols < limit;) {
                    Request *c = reqs.at(*it).get();
                    const int64_t cc = c->kk + c->q;
                    const int64_t nb = request_bytes(gp->n, (int32_t)(cols + cc));
                    if (c->graph == r->graph && (c->kk > 0) == (r->kk > 0) && cols + cc <= limit &&
                        graph_bytes + inflight_bytes + nb <= budget) {
                        batch.push_back(c);
                        cols += cc;
                        batch_bytes = nb;
                        it = queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                inflight_bytes += batch_bytes;
                peak_inflight_bytes = std::max(peak_inflight_bytes, inflight_bytes);
                in_flight += (int)batch.size();
                max_in_flight = std::max(max_in_flight, in_flight);
                max_batch = std::max(max_batch, (int)batch.size());
                const Clock::time_point now = Clock::now();
                for (Request *b : batch) b->t_admit = now;
            }
            lap_status_t st;
            try {
                const Graph &g = *gp;
                std::vector<cfc::SampledQuery> qs;
                for (Request *b : batch) qs.push_back({b->kk, b->seed, b->q, b->nodes.data(), b->far.data()});
                const bool resident = batch[0]->kk == 0;
                st = cfc::farness_sampled_batch(g.h, qs.data(), (int)qs.size(), resident ? g.xs.get() : nullptr,
                                                resident ? g.piv.get() : nullptr, resident ? g.kp : 0, g.opts, s);
                cfc::release_workspace(g.h, s);  // back to the pool, for the next admission
                cudaError_t e = cudaStreamSynchronize(s);
                if (e != cudaSuccess && st == LAP_OK) st = LAP_ECUDA;
            } catch (const cfc::Error &e) {
                cfc::set_last_error(e.what);
                cudaStreamSynchronize(s);
                st = e.status;
            } catch (const std::bad_alloc &) {
                st = LAP_ENOMEM;
            } catch (...) {
                st = LAP_ECUDA;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                const Clock::time_point now = Clock::now();
                inflight_bytes -= batch_bytes;
                in_flight -= (int)batch.size();
                for (Request *r : batch) {
                    r->status = st;
                    r->t_done = now;
                    r->done = true;
                    if (st == LAP_OK) {
                        lat_ms.push_back(ms_between(r->t_submit, r->t_done));
                        ++completed;
                        rhs_done += r->kk + r->q;  // resident requests: kk = 0, their q columns
                        span1 = r->t_done;
                    }
                }
            }
            cv_done.notify_all();
            cv_work.notify_all();  // memory came back: the next request may fit
        }
    }
};

extern "C" {

void cfc_server_default_opts(cfc_server_opts_t *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->slots = 4;
    o->hbm_budget = 0;
    o->batch_columns = 1024;
    lap_default_solve_opts(&o->solve);
}

lap_status_t cfc_server_create(const cfc_server_opts_t *o, cfc_server_t **out) {
    return cfc::guard([&]() -> lap_status_t {
        CFC_REQUIRE(o && out, LAP_EINVAL, "NULL argument");
        CFC_REQUIRE(o->slots >= 1 && o->slots <= 64, LAP_EINVAL, "need 1 <= slots <= 64");
        CFC_REQUIRE(o->hbm_budget >= 0, LAP_EINVAL, "hbm_budget must be >= 0");
        CFC_REQUIRE(o->batch_columns >= 0, LAP_EINVAL, "batch_columns must be >= 0");
        *out = nullptr;
        auto sv = std::make_unique<cfc_server>();
        sv->o = *o;
        CFC_CUDA(cudaGetDevice(&sv->device));
        size_t fr = 0, tot = 0;
        CFC_CUDA(cudaMemGetInfo(&fr, &tot));
        sv->budget = o->hbm_budget > 0 ? o->hbm_budget : (int64_t)(0.8 * (double)fr);
        for (int i = 0; i <= o->slots; ++i) {
            cudaStream_t s;
            CFC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            if (i < o->slots)
                sv->streams.push_back(s);
            else
                sv->admin = s;
        }
        cfc_server *p = sv.get();
        for (int i = 0; i < o->slots; ++i) p->workers.emplace_back([p, i] { p->worker(i); });
        *out = sv.release();
        return LAP_OK;
    });
}

lap_status_t cfc_server_add_graph(cfc_server_t *sv, int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                  const double *w, int32_t *graph_id) {
    return cfc::guard([&]() -> lap_status_t {
        CFC_REQUIRE(sv && graph_id, LAP_EINVAL, "NULL argument");
        cfc_server::Graph g;
        lap_hier_opts_t ho;
        lap_default_hier_opts(&ho);
        ho.eager = 1;  // every level now: requests never grow the hierarchy
        std::lock_guard<std::mutex> admin_lk(sv->admin_mu);
        cudaStream_t s = sv->admin;
        lap_status_t st = lap_build_hierarchy(n, m, src, dst, w, &ho, s, &g.h);
        if (st != LAP_OK) return st;
        std::unique_ptr<lap_hierarchy, void (*)(lap_hierarchy *)> guard_h(g.h, lap_hierarchy_destroy);
        g.n = n;
        // tune once on a request-shaped solve, then pin what was chosen
        const int32_t kk = (int32_t)std::min<int64_t>(200, n), q = (int32_t)std::min<int64_t>(16, n);
        std::vector<int32_t> nodes(q);
        for (int i = 0; i < q; ++i) nodes[i] = (int32_t)((int64_t)i * n / q);
        std::vector<double> f(q);
        lap_solve_info_t info{};
        st = cfc::farness_sampled(g.h, kk, 0, q, nodes.data(), f.data(), sv->o.solve, s, &info);
        cfc::release_workspace(g.h, s);
        CFC_CUDA(cudaStreamSynchronize(s));
        if (st != LAP_OK) return st;
        g.opts = sv->o.solve;
        g.opts.k_tile = info.k_tile;
        g.opts.levels_used = info.levels_used;
        g.opts.nu_coarse = info.nu_coarse;
        g.opts.cycle = info.cycle;
        g.opts.coarse_scale = info.coarse_scale;
        g.opts.w_levels = info.w_levels;
        g.bytes = cfc::hierarchy_bytes(g.h);  // with any BF16 copies the tuning made
        int32_t id;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            id = (int32_t)sv->graphs.size();
        }
        if (sv->o.resident_pivots > 0) {
            g.kp = (int32_t)std::min<int64_t>(std::min<int64_t>(sv->o.resident_pivots, n), 4096);
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                CFC_REQUIRE(sv->graph_bytes + sv->inflight_bytes + g.bytes + n * g.kp * 8 <= sv->budget,
                            LAP_EBUDGET, "graph and its pivot solutions do not fit the HBM budget");
            }
            g.piv.alloc_persistent(g.kp);
            g.xs.alloc_persistent((size_t)n * g.kp);
            st = cfc::pivot_solutions(g.h, g.kp, sv->o.pivot_seed + (uint64_t)id, g.xs.get(), g.piv.get(), g.opts,
                                      s, nullptr);
            cfc::release_workspace(g.h, s);
            CFC_CUDA(cudaStreamSynchronize(s));
            if (st != LAP_OK) return st;
            g.bytes += n * g.kp * 8 + g.kp * 4;
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        CFC_REQUIRE(sv->graph_bytes + sv->inflight_bytes + g.bytes <= sv->budget, LAP_EBUDGET,
                    "graph does not fit the HBM budget");
        CFC_REQUIRE((int32_t)sv->graphs.size() == id, LAP_EINVAL, "graphs added concurrently");
        sv->graph_bytes += g.bytes;
        *graph_id = id;
        sv->graphs.push_back(std::move(g));
        guard_h.release();
        return LAP_OK;
    });
}

lap_status_t cfc_server_submit(cfc_server_t *sv, int32_t graph_id, int32_t q, const int32_t *nodes,
                               int32_t n_pivots, uint64_t seed, int64_t *request_id) {
    return cfc::guard([&]() -> lap_status_t {
        CFC_REQUIRE(sv && nodes && request_id, LAP_EINVAL, "NULL argument");
        auto r = std::make_unique<cfc_server::Request>();
        std::unique_lock<std::mutex> lk(sv->mu);
        CFC_REQUIRE(graph_id >= 0 && graph_id < (int32_t)sv->graphs.size(), LAP_EINVAL, "unknown graph id");
        const cfc_server::Graph &g = sv->graphs[graph_id];
        CFC_REQUIRE(q >= 1 && q <= g.n, LAP_EINVAL, "need 1 <= q <= n");
        CFC_REQUIRE(n_pivots >= 0 && n_pivots <= g.n, LAP_EINVAL, "need 0 <= n_pivots <= n");
        CFC_REQUIRE(n_pivots > 0 || g.kp > 0, LAP_EINVAL, "n_pivots = 0 needs the graph's resident pivot set");
        CFC_REQUIRE(n_pivots + q <= 4096, LAP_EBUDGET, "n_pivots + q must be <= 4096 columns");
        for (int i = 0; i < q; ++i) CFC_REQUIRE(nodes[i] >= 0 && nodes[i] < g.n, LAP_EINVAL, "query node out of range");
        r->graph = graph_id;
        r->q = q;
        r->kk = n_pivots;
        r->seed = seed;
        r->nodes.assign(nodes, nodes + q);
        r->far.assign(q, 0.0);
        r->bytes = cfc_server::request_bytes(g.n, n_pivots + q);
        CFC_REQUIRE(sv->graph_bytes + r->bytes <= sv->budget, LAP_EBUDGET,
                    "request does not fit the HBM budget beside the resident graphs");
        r->id = sv->next_id++;
        r->t_submit = Clock::now();
        if (!sv->have_span) {
            sv->have_span = true;
            sv->span0 = r->t_submit;
        }
        ++sv->submitted;
        *request_id = r->id;
        sv->queue.push_back(r->id);
        sv->reqs.emplace(r->id, std::move(r));
        lk.unlock();
        sv->cv_work.notify_all();
        return LAP_OK;
    });
}

lap_status_t cfc_server_poll(cfc_server_t *sv, int64_t request_id, int32_t wait_ms, double *farness,
                             cfc_request_info_t *info) {
    return cfc::guard([&]() -> lap_status_t {
        CFC_REQUIRE(sv, LAP_EINVAL, "NULL argument");
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->reqs.find(request_id);
        CFC_REQUIRE(it != sv->reqs.end(), LAP_EINVAL, "unknown or already polled request id");
        cfc_server::Request *r = it->second.get();
        auto ready = [&] { return r->done; };
        if (wait_ms < 0)
            sv->cv_done.wait(lk, ready);
        else if (wait_ms > 0)
            sv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
        if (!r->done) return LAP_EPENDING;
        if (farness) std::memcpy(farness, r->far.data(), r->far.size() * sizeof(double));
        if (info) {
            info->status = r->status;
            info->graph_id = r->graph;
            info->q = r->q;
            info->n_pivots = r->kk;
            info->device_bytes = r->bytes;
            info->queue_ms = ms_between(r->t_submit, r->t_admit);
            info->run_ms = ms_between(r->t_admit, r->t_done);
            info->latency_ms = ms_between(r->t_submit, r->t_done);
        }
        const lap_status_t st = r->status;
        sv->reqs.erase(it);
        return st;
    });
}

lap_status_t cfc_server_stats(cfc_server_t *sv, cfc_server_stats_t *out) {
    return cfc::guard([&]() -> lap_status_t {
        CFC_REQUIRE(sv && out, LAP_EINVAL, "NULL argument");
        std::lock_guard<std::mutex> lk(sv->mu);
        std::memset(out, 0, sizeof(*out));
        out->submitted = sv->submitted;
        out->completed = sv->completed;
        out->pending = (int64_t)sv->queue.size();
        out->in_flight = sv->in_flight;
        out->max_in_flight = sv->max_in_flight;
        out->graph_bytes = sv->graph_bytes;
        out->budget_bytes = sv->budget;
        out->peak_in_flight_bytes = sv->peak_inflight_bytes;
        out->max_batch = sv->max_batch;
        if (!sv->lat_ms.empty()) {
            std::vector<double> v = sv->lat_ms;
            std::sort(v.begin(), v.end());
            // nearest rank: the smallest value with at least p% of the values at or below it
            auto rank = [&](double p) {
                size_t i = (size_t)std::ceil(p / 100.0 * (double)v.size());
                return v[std::min(v.size(), std::max<size_t>(i, 1)) - 1];
            };
            out->p50_ms = rank(50.0);
            out->p99_ms = rank(99.0);
            out->max_ms = v.back();
            double t = 0;
            for (double x : v) t += x;
            out->mean_ms = t / (double)v.size();
            const double span_s = ms_between(sv->span0, sv->span1) / 1e3;
            if (span_s > 0) {
                out->queries_per_s = (double)sv->completed / span_s;
                out->rhs_per_s = (double)sv->rhs_done / span_s;
            }
        }
        return LAP_OK;
    });
}

void cfc_server_reset_stats(cfc_server_t *sv) {
    if (!sv) return;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->lat_ms.clear();
    sv->completed = sv->rhs_done = 0;
    sv->submitted = (int64_t)sv->queue.size() + sv->in_flight;
    sv->max_in_flight = sv->in_flight;
    sv->max_batch = 0;
    sv->peak_inflight_bytes = sv->inflight_bytes;
    sv->have_span = false;
    if (!sv->queue.empty() || sv->in_flight > 0) {
        sv->have_span = true;
        sv->span0 = Clock::now();
    }
}

void cfc_server_destroy(cfc_server_t *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;  // queued requests are dropped; those in flight finish
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    for (auto &g : sv->graphs) lap_hierarchy_destroy(g.h);
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    if (sv->admin) cudaStreamDestroy(sv->admin);
    delete sv;
}

}  // extern "C"
