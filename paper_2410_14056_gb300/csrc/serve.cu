// Serving loop: SC queries on resident graphs with continuous batching.
//
// A submitted request is queued for a pool of planner threads, which compute
// its scheduled plan on the host.  A worker thread owns a non-blocking
// stream; it admits planned requests while the device memory they need and
// the number of requests on the GPU fit the configured limits (uploading
// each and preparing its edges),
// then runs iterations: each iteration is one persistent counting launch over
// a window of tasks of every admitted request.  A request whose last tasks
// were launched is finalized and its results copied back on a second stream;
// the worker sees completion through an event, releases its memory and wakes
// its waiter.  Newly submitted requests join at the next iteration.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "internal.h"

namespace bq {
namespace {

using Clock = std::chrono::steady_clock;

// Device layout of a request with k edges (byte offsets; 256-aligned
// sections).  Inputs, uploaded by one copy: descriptor | uv[2k] | tau[k] |
// nwalks[k].  Work: info[k] | tasks[k] | begin[k + 1].
// Outputs, read back by one copy: status word (16 B) | counts[4k] | sc[k].
struct Layout {
    size_t qd, uv, tau, nw, in_bytes;
    size_t info, tasks, begin;
    size_t out, counts, sc, out_bytes;
    size_t total;
};

Layout layout_of(uint64_t k) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    Layout L;
    size_t p = 0;
    L.qd = p;
    p += up(sizeof(QueryDesc));
    L.uv = p;
    p += up(8 * k);
    L.tau = p;
    p += up(4 * k);
    L.nw = p;
    p += up(4 * k);
    L.in_bytes = p;
    L.info = p;
    p += up(sizeof(BInfo) * k);
    L.tasks = p;
    p += up(4 * k);
    L.begin = p;
    p += up(8 * (k + 1));
    L.out = p;
    L.counts = p + 16;
    L.sc = L.counts + 16 * k;
    L.out_bytes = 16 + 24 * k;
    p += up(L.out_bytes);
    L.total = p;
    return L;
}

struct Request {
    uint64_t id = 0;
    uint32_t graph = 0;
    uint64_t k = 0;
    double eps = 0.1;
    uint64_t seed = 0;
    Layout L;
    Clock::time_point t_submit, t_done;
    int status = BQ_OK;
    std::string error;  // message of a failed request
    // the pairs as submitted, until a planner moves them into h_in
    std::vector<uint32_t> uv_in;
    // pinned host image of the input sections (pairs and plan, written by a
    // planner thread; the descriptor is written at admission), uploaded by
    // one asynchronous copy and returned to the pool when the request ends
    char *h_in = nullptr;
    size_t h_in_cap = 0;
    double walk_steps = 0;
    uint64_t tasks_total = 0, tasks_launched = 0;
    // device
    char *dbuf = nullptr;
    size_t dbytes = 0;
    cudaEvent_t fin_ev = nullptr;   // finalize done on the compute stream
    cudaEvent_t done_ev = nullptr;  // results in h_out (copy stream)
    bool finalizing = false;
    // pinned host image of the output sections (from the server's pool;
    // returned when the waiter has copied it out)
    char *h_out = nullptr;
    size_t h_out_cap = 0;

    QueryDesc *d_qd() const { return reinterpret_cast<QueryDesc *>(dbuf + L.qd); }
    BInfo *d_info() const { return reinterpret_cast<BInfo *>(dbuf + L.info); }
    uint64_t *d_begin() const { return reinterpret_cast<uint64_t *>(dbuf + L.begin); }
    uint32_t *h_uv() { return reinterpret_cast<uint32_t *>(h_in + L.uv); }
    uint32_t *h_tau() { return reinterpret_cast<uint32_t *>(h_in + L.tau); }
    uint32_t *h_nw() { return reinterpret_cast<uint32_t *>(h_in + L.nw); }
};

using RequestPtr = std::shared_ptr<Request>;

size_t request_bytes(uint64_t k) { return layout_of(k).total; }

// Pinned host blocks for result images, reused by size class (powers of two
// from 4 KiB), so that results come back by asynchronous DMA.  Blocks are
// allocated on the worker thread and returned by waiters.
struct PinnedPool {
    // Blocks come from per-size-class free lists, then from one page-locked
    // arena allocated when the server starts (so that a request does not wait
    // for page locking), then from cudaMallocHost.
    std::mutex mu;
    std::unordered_map<size_t, std::vector<char *>> free;
    std::vector<char *> all;
    char *arena = nullptr;
    size_t arena_size = 0, arena_used = 0;
    uint64_t fallbacks = 0;  // blocks from cudaMallocHost after the arena ran out
    double fallback_s = 0;   // and the time those calls took
    static size_t size_class(size_t bytes) {
        size_t c = 4096;
        while (c < bytes) c <<= 1;
        return c;
    }
    int reserve(size_t bytes) {
        if (bytes == 0) return BQ_OK;
        if (cudaMallocHost((void **)&arena, bytes) != cudaSuccess) {
            cudaGetLastError();
            arena = nullptr;
            return fail(BQ_ENOMEM, "cannot page-lock %zu bytes of host memory for the server", bytes);
        }
        arena_size = bytes;
        return BQ_OK;
    }
    char *get(size_t bytes, size_t &cap) {
        cap = size_class(bytes);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto &v = free[cap];
            if (!v.empty()) {
                char *p = v.back();
                v.pop_back();
                return p;
            }
            if (arena && arena_used + cap <= arena_size) {
                char *p = arena + arena_used;
                arena_used += cap;
                return p;
            }
        }
        char *p = nullptr;
        const auto t0 = std::chrono::steady_clock::now();
        if (cudaMallocHost((void **)&p, cap) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        std::lock_guard<std::mutex> lk(mu);
        all.push_back(p);
        ++fallbacks;
        fallback_s += dt;
        return p;
    }
    void put(char *p, size_t cap) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        free[cap].push_back(p);
    }
    void release() {
        for (char *p : all) cudaFreeHost(p);
        if (arena) cudaFreeHost(arena);
        arena = nullptr;
        arena_size = arena_used = 0;
        all.clear();
        free.clear();
    }
};

}  // namespace
}  // namespace bq

struct bq_server {
    std::vector<bq_graph *> graphs;
    bq_server_config cfg;
    bq::Sampler smp{0, 0, 1};
    int device = 0;
    int lanes = 4;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    // iteration descriptors: pinned host ring and device ring
    static constexpr int kRing = 4;  // iterations the worker may run ahead of the GPU
    bq::ServeItem *h_items[kRing] = {};
    bq::ServeItem *d_items[kRing] = {};
    unsigned long long *d_counter = nullptr;
    cudaEvent_t ring_ev[kRing] = {};
    bool ring_used[kRing] = {};
    int ring_next = 0;
    uint32_t *status = nullptr;
    bq::PinnedPool pinned;
    std::vector<cudaEvent_t> events;  // free events (worker thread only)

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<bq::RequestPtr> to_plan;  // submitted, waiting for a planner thread
    uint32_t planning = 0;                // requests being planned now
    std::condition_variable cv_plan;
    std::vector<std::thread> planners;
    std::deque<bq::RequestPtr> pending;   // planned, waiting for admission
    std::vector<bq::RequestPtr> inflight;
    std::unordered_map<uint64_t, bq::RequestPtr> done;
    std::unordered_set<uint64_t> live;  // submitted and not yet returned by bq_server_wait
    uint64_t next_id = 1;
    uint64_t held_bytes = 0;
    bool stop = false;
    std::thread worker;

    // statistics
    bq::Clock::time_point t_start;
    uint64_t submitted = 0, completed = 0, failed = 0, edges_completed = 0, iterations = 0;
    double walk_steps = 0;
    double t_admit = 0, t_launch = 0, t_complete = 0, t_idle = 0;  // worker seconds per phase
    double t_plan = 0, t_plan_max = 0;  // planner seconds: all requests, the longest one
    std::vector<double> latencies_ms;
};

namespace bq {
namespace {

uint32_t bouquet_of(const bq_server *srv) { return 32u * (uint32_t)srv->lanes; }

// Events are reused (worker thread only).
cudaEvent_t take_event(bq_server *srv) {
    if (!srv->events.empty()) {
        cudaEvent_t e = srv->events.back();
        srv->events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void give_event(bq_server *srv, cudaEvent_t &e) {
    if (e) srv->events.push_back(e);
    e = nullptr;
}

// Plan pairs [lo, hi) of a request: tau and N per pair from the endpoint
// degrees (the scheduled plan), the bouquet tasks and walk steps summed.
// Returns the index of the first pair that cannot be planned (hi if none),
// with its code and message.
struct PlanPart {
    uint64_t bad = 0;
    int code = BQ_OK;
    std::string msg;
    uint64_t tasks = 0;
    double steps = 0.0;
};

void plan_range(const bq_graph *g, const uint32_t *edges_uv, uint64_t lo, uint64_t hi, double eps,
                const bq_schedule &sched, uint32_t bouquet, uint32_t *tau, uint32_t *nw, PlanPart &out) {
    const int64_t *off = g->h_offsets.data();
    out.bad = hi;
    // the endpoints' offsets are random reads into an array of up to
    // several hundred MB: request them kAhead pairs before they are used
    constexpr uint64_t kAhead = 32;
    for (uint64_t i = lo; i < hi && i < lo + kAhead; ++i) {
        if (edges_uv[2 * i] < g->n) __builtin_prefetch(off + edges_uv[2 * i]);
        if (edges_uv[2 * i + 1] < g->n) __builtin_prefetch(off + edges_uv[2 * i + 1]);
    }
    char buf[160];
    for (uint64_t i = lo; i < hi; ++i) {
        if (i + kAhead < hi) {
            const uint32_t pa = edges_uv[2 * (i + kAhead)], pb = edges_uv[2 * (i + kAhead) + 1];
            if (pa < g->n) __builtin_prefetch(off + pa);
            if (pb < g->n) __builtin_prefetch(off + pb);
        }
        const uint32_t a = edges_uv[2 * i], b = edges_uv[2 * i + 1];
        int64_t da = 0, db = 0;
        if (a < g->n && b < g->n && a != b) {
            da = off[a + 1] - off[a];
            db = off[b + 1] - off[b];
        }
        if (da == 0 || db == 0) {
            snprintf(buf, sizeof buf, "pair %llu: (%u, %u) is not an edge", (unsigned long long)i, a, b);
            out.bad = i;
            out.code = BQ_ENOEDGE;
            out.msg = buf;
            return;
        }
        const double s_e = 1.0 / (double)da + 1.0 / (double)db;
        uint32_t t = 1;
        double n = 0.0;
        plan_scheduled_edge(s_e, eps, sched, t, n);
        if (n < 1.0) n = 1.0;
        if (n * 2.0 * (double)t >= 4294967296.0) {
            snprintf(buf, sizeof buf, "pair %llu: 2 N tau = %.3g reaches 2^32", (unsigned long long)i,
                     n * 2.0 * (double)t);
            out.bad = i;
            out.code = BQ_EOVERFLOW;
            out.msg = buf;
            return;
        }
        tau[i] = t;
        nw[i] = (uint32_t)n;
        out.tasks += 2ull * ((nw[i] + bouquet - 1) / bouquet);
        out.steps += 2.0 * (double)nw[i] * (double)t;
    }
}

// Requests with at least kPlanSplit pairs are planned by up to kPlanThreads
// threads, one contiguous range each; the error reported is always that of
// the lowest failing pair, as in one pass.
constexpr uint64_t kPlanSplit = 32768;
constexpr unsigned kPlanThreads = 4;

// Plan one request on the host (a planner thread, no lock): fill tau and N
// per edge of its input image from the endpoint degrees (the scheduled
// plan), count its bouquet tasks and walk steps.  A pair with an endpoint of
// degree 0 fails here (BQ_ENOEDGE), as does 2 N tau >= 2^32 (BQ_EOVERFLOW);
// whether a pair is an edge is checked on the GPU (the prepare kernel's row
// search), whose status comes back with the results.
int plan_request(bq_server *srv, Request &r) {
    const bq_graph *g = srv->graphs[r.graph];
    r.h_in = srv->pinned.get(r.L.in_bytes, r.h_in_cap);
    if (!r.h_in) return fail(BQ_ENOMEM, "server: no pinned host memory for a request");
    if (r.k) memcpy(r.h_uv(), r.uv_in.data(), 8 * r.k);
    std::vector<uint32_t>().swap(r.uv_in);
    const uint32_t *edges_uv = r.h_uv();
    const bq_schedule sched{srv->cfg.tau_scale, srv->cfg.tau_add, srv->cfg.tau_max,
                            srv->cfg.n_scale,   srv->cfg.n_min,   0};
    const uint32_t bouquet = bouquet_of(srv);
    uint32_t *tau = r.h_tau(), *nw = r.h_nw();
    unsigned parts = 1;
    if (r.k >= kPlanSplit)
        parts = (unsigned)std::min<uint64_t>(kPlanThreads, r.k / (kPlanSplit / 2));
    std::vector<PlanPart> out(parts);
    const uint64_t per = (r.k + parts - 1) / parts;
    auto run = [&](unsigned i) {
        const uint64_t lo = std::min<uint64_t>(r.k, (uint64_t)i * per), hi = std::min<uint64_t>(r.k, lo + per);
        plan_range(g, edges_uv, lo, hi, r.eps, sched, bouquet, tau, nw, out[i]);
    };
    if (parts == 1) {
        run(0);
    } else {
        std::vector<std::thread> pool;
        for (unsigned i = 1; i < parts; ++i) pool.emplace_back(run, i);
        run(0);
        for (auto &t : pool) t.join();
    }
    r.tasks_total = 0;
    r.walk_steps = 0;
    for (const PlanPart &p : out) {  // parts in pair order: the first error is the lowest pair's
        if (p.code != BQ_OK) return fail(p.code, "%s", p.msg.c_str());
        r.tasks_total += p.tasks;
        r.walk_steps += p.steps;
    }
    return BQ_OK;
}

// Allocate, upload and prepare one planned request (worker thread, no lock).
int admit(bq_server *srv, Request &r) {
    const bq_graph *g = srv->graphs[r.graph];
    cudaStream_t s = srv->stream;
    cudaError_t e = cudaMallocAsync((void **)&r.dbuf, r.dbytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        r.dbuf = nullptr;
        return fail(BQ_ENOMEM, "server: cannot allocate %zu bytes for a request", r.dbytes);
    }
    QueryDesc qd;
    qd.g = graph_desc(g);
    qd.seed = r.seed;
    qd.uv = reinterpret_cast<const uint32_t *>(r.dbuf + r.L.uv);
    qd.tau = reinterpret_cast<const uint32_t *>(r.dbuf + r.L.tau);
    qd.nwalks = reinterpret_cast<const uint32_t *>(r.dbuf + r.L.nw);
    qd.counts = reinterpret_cast<uint32_t *>(r.dbuf + r.L.counts);
    qd.sc = reinterpret_cast<double *>(r.dbuf + r.L.sc);
    qd.k = r.k;
    qd.ebase = 0;
    memcpy(r.h_in + r.L.qd, &qd, sizeof(qd));
    e = cudaMemcpyAsync(r.dbuf, r.h_in, r.L.in_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r.dbuf + r.L.out, 0, 16, s);
    if (e != cudaSuccess) return cuda_fail(e, "server: request upload");
    r.fin_ev = take_event(srv);
    r.done_ev = take_event(srv);
    if (!r.fin_ev || !r.done_ev) return fail(BQ_ECUDA, "server: cannot create events");
    return BQ_OK;  // prepared with the rest of its admission pass (prepare_pass)
}

// The requests' slots in a multi-request launch list.
void add_to_list(ServeMany &L, Request &r) {
    const uint32_t j = L.m++;
    L.qd[j] = r.d_qd();
    L.info[j] = r.d_info();
    L.tasks[j] = reinterpret_cast<uint32_t *>(r.dbuf + r.L.tasks);
    L.begin[j] = r.d_begin();
    L.status[j] = reinterpret_cast<uint32_t *>(r.dbuf + r.L.out);
    L.edge_base[j + 1] = L.edge_base[j] + r.k;
}

// Edge info, task counts and task prefix of a pass's admitted requests: two
// launches per kServeMany requests instead of several per request.
int prepare_pass(bq_server *srv, const std::vector<Request *> &reqs) {
    ServeMany L{};
    for (size_t i = 0; i < reqs.size(); ++i) {
        add_to_list(L, *reqs[i]);
        if (L.m == kServeMany || i + 1 == reqs.size()) {
            const int rc = serve_prepare_many(L, bouquet_of(srv), srv->stream);
            if (rc) return rc;
            L = ServeMany{};
        }
    }
    return BQ_OK;
}

// Finalize on the compute stream; the copy stream then brings the output
// section back into a pinned block and frees the request's device memory,
// so the compute stream goes on with other requests meanwhile.
void finish_copy(bq_server *srv, Request &r) {
    cudaEventRecord(r.fin_ev, srv->stream);
    r.h_out = srv->pinned.get(r.L.out_bytes, r.h_out_cap);
    cudaStreamWaitEvent(srv->copy_stream, r.fin_ev, 0);
    if (r.h_out)
        cudaMemcpyAsync(r.h_out, r.dbuf + r.L.out, r.L.out_bytes, cudaMemcpyDeviceToHost, srv->copy_stream);
    cudaFreeAsync(r.dbuf, srv->copy_stream);
    r.dbuf = nullptr;
    cudaEventRecord(r.done_ev, srv->copy_stream);
    r.finalizing = true;
}

// Finalize a set of requests (one launch per kServeMany), then start each
// one's result copy.
void finalize_many(bq_server *srv, const std::vector<Request *> &reqs) {
    ServeMany L{};
    size_t first = 0;
    for (size_t i = 0; i < reqs.size(); ++i) {
        add_to_list(L, *reqs[i]);
        if (L.m == kServeMany || i + 1 == reqs.size()) {
            serve_finalize_many(L, srv->stream);
            for (size_t j = first; j <= i; ++j) finish_copy(srv, *reqs[j]);
            first = i + 1;
            L = ServeMany{};
        }
    }
}

// One iteration: a window of tasks of every admitted request, one launch.
// Returns false when no request has tasks left to launch.
bool iterate(bq_server *srv) {
    NvtxRange nvtx_range("bq_server_iteration");
    std::vector<Request *> active;
    for (auto &r : srv->inflight)
        if (!r->finalizing && r->tasks_launched < r->tasks_total) active.push_back(r.get());
    if (active.empty()) return false;
    // The window grows with the backlog (half of the tasks left, at most 8
    // configured windows): a busy server amortises each launch over more work,
    // a lightly loaded one keeps iterations short for latency.
    uint64_t remaining = 0;
    for (Request *r : active) remaining += r->tasks_total - r->tasks_launched;
    const uint64_t window = srv->cfg.tasks_per_iteration;
    const uint64_t budget = std::min(std::max(window, remaining / 2), 8 * window);
    std::vector<uint64_t> take(active.size(), 0);
    uint64_t used = 0;
    // fair share, then hand what is left to requests that still have tasks
    for (int pass = 0; pass < 2 && used < budget; ++pass) {
        uint64_t open = 0;
        for (size_t i = 0; i < active.size(); ++i)
            if (active[i]->tasks_total - active[i]->tasks_launched > take[i]) ++open;
        if (!open) break;
        const uint64_t share = std::max<uint64_t>(1, (budget - used) / open);
        for (size_t i = 0; i < active.size() && used < budget; ++i) {
            const uint64_t left = active[i]->tasks_total - active[i]->tasks_launched - take[i];
            const uint64_t w = std::min(std::min(left, share), budget - used);
            take[i] += w;
            used += w;
        }
    }
    const int slot = srv->ring_next;
    if (srv->ring_used[slot]) cudaEventSynchronize(srv->ring_ev[slot]);
    ServeItem *items = srv->h_items[slot];
    uint32_t n = 0;
    uint64_t base = 0;
    for (size_t i = 0; i < active.size(); ++i) {
        if (!take[i]) continue;
        Request &r = *active[i];
        items[n].qd = r.d_qd();
        items[n].info = r.d_info();
        items[n].begin = r.d_begin();
        items[n].k = r.k;
        items[n].task_lo = r.tasks_launched;
        items[n].item_base = base;
        base += take[i];
        r.tasks_launched += take[i];
        ++n;
    }
    cudaMemcpyAsync(srv->d_items[slot], items, sizeof(ServeItem) * n, cudaMemcpyHostToDevice, srv->stream);
    serve_iterate(srv->d_items[slot], n, base, srv->lanes, srv->smp, srv->d_counter, srv->stream);
    cudaEventRecord(srv->ring_ev[slot], srv->stream);
    srv->ring_used[slot] = true;
    srv->ring_next = (slot + 1) % bq_server::kRing;
    std::vector<Request *> finished;
    for (Request *r : active)
        if (r->tasks_launched == r->tasks_total) finished.push_back(r);
    finalize_many(srv, finished);
    ++srv->iterations;
    return true;
}

// Hand finished requests to their waiters.  With `block`, wait for the
// oldest finalizing request first (nothing else to launch meanwhile).
void poll_completions(bq_server *srv, bool block) {
    std::vector<RequestPtr> finished;
    for (auto &r : srv->inflight) {
        if (!r->finalizing) continue;
        const cudaError_t e =
            block && finished.empty() ? cudaEventSynchronize(r->done_ev) : cudaEventQuery(r->done_ev);
        if (e == cudaErrorNotReady) continue;
        uint32_t bits = 0;
        if (e == cudaSuccess && r->h_out) memcpy(&bits, r->h_out, sizeof(bits));
        if (e != cudaSuccess) {
            r->status = BQ_ECUDA;
            r->error = cudaGetErrorString(e);
        } else if (!r->h_out) {
            r->status = BQ_ENOMEM;
            r->error = "no pinned host memory for the results";
        } else if (bits & kStatusNoEdge) {
            r->status = BQ_ENOEDGE;
            r->error = "a queried pair is not an edge";
        } else if (bits) {
            r->status = BQ_EOVERFLOW;
            r->error = "a plan entry is out of range";
        }
        finished.push_back(r);
    }
    if (finished.empty()) return;
    std::lock_guard<std::mutex> lk(srv->mu);
    const auto now = Clock::now();
    for (auto &r : finished) {
        give_event(srv, r->fin_ev);
        give_event(srv, r->done_ev);
        srv->pinned.put(r->h_in, r->h_in_cap);  // its upload finished long before
        r->h_in = nullptr;
        if (r->status != BQ_OK) {  // nothing to read: the block goes back now
            srv->pinned.put(r->h_out, r->h_out_cap);
            r->h_out = nullptr;
        }
        srv->held_bytes -= r->dbytes;
        r->t_done = now;
        if (r->status != BQ_OK) {
            ++srv->failed;
        } else {
            ++srv->completed;
            srv->edges_completed += r->k;
            srv->walk_steps += r->walk_steps;
        }
        srv->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        srv->inflight.erase(std::find(srv->inflight.begin(), srv->inflight.end(), r));
        srv->done[r->id] = r;
    }
    srv->cv_done.notify_all();
}

}  // namespace
}  // namespace bq

namespace bq {
namespace {

// A request that could not be planned or admitted completes at once with its
// error status (its memory, if any, is released).
void complete_failed(bq_server *srv, const RequestPtr &r, int status) {
    if (r->dbuf) {
        // a failed admission may have its upload in flight: let it finish
        // before the pinned image goes back to the pool (a rare path)
        cudaStreamSynchronize(srv->stream);
        cudaFreeAsync(r->dbuf, srv->stream);
        r->dbuf = nullptr;
    }
    give_event(srv, r->fin_ev);
    give_event(srv, r->done_ev);
    srv->pinned.put(r->h_in, r->h_in_cap);
    r->h_in = nullptr;
    const char *msg = bq_last_error();
    std::lock_guard<std::mutex> lk(srv->mu);
    r->status = status;
    r->error = msg ? msg : "";
    r->t_done = Clock::now();
    if (r->dbytes) srv->held_bytes -= r->dbytes;
    r->dbytes = 0;
    ++srv->failed;
    srv->done[r->id] = r;
    srv->cv_done.notify_all();
}

// Planner thread: plans submitted requests (host work proportional to their
// edges) and hands them to the worker; a request that cannot be planned is
// completed at once with its error.
void planner_main(bq_server *srv) {
    cudaSetDevice(srv->device);
    for (;;) {
        RequestPtr r;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_plan.wait(lk, [srv] { return srv->stop || !srv->to_plan.empty(); });
            if (srv->to_plan.empty()) return;  // stopping, and nothing left to plan
            r = srv->to_plan.front();
            srv->to_plan.pop_front();
            ++srv->planning;
        }
        clear_error();
        const auto t0 = Clock::now();
        const int rc = plan_request(srv, *r);
        const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
        const std::string msg = rc != BQ_OK ? std::string(bq_last_error()) : std::string();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            --srv->planning;
            srv->t_plan += dt;
            if (dt > srv->t_plan_max) srv->t_plan_max = dt;
            if (rc == BQ_OK) {
                srv->pending.push_back(r);
            } else {
                srv->pinned.put(r->h_in, r->h_in_cap);
                r->h_in = nullptr;
                r->status = rc;
                r->error = msg;
                r->t_done = Clock::now();
                ++srv->failed;
                srv->done[r->id] = r;
                srv->cv_done.notify_all();
            }
        }
        srv->cv_work.notify_one();
    }
}

// Requests admitted per pass while others are on the GPU, so that a burst
// of arrivals does not hold back the next iteration's launch.
constexpr size_t kAdmitPerPass = 8;

void worker_main(bq_server *srv) {
    cudaSetDevice(srv->device);
    const uint64_t budget = srv->cfg.device_budget_bytes;
    auto lap = [](Clock::time_point &t0) {
        const auto t1 = Clock::now();
        const double s = std::chrono::duration<double>(t1 - t0).count();
        t0 = t1;
        return s;
    };
    for (;;) {
        // admission: FIFO, while slots and device memory allow
        std::vector<RequestPtr> admitted;
        bool idle = false;
        auto t0 = Clock::now();
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                if (srv->pending.empty()) break;
                if (!srv->inflight.empty() && admitted.size() >= kAdmitPerPass) break;
                RequestPtr r = srv->pending.front();
                const size_t bytes = request_bytes(r->k);
                if (bytes > budget) {
                    srv->pending.pop_front();
                    lk.unlock();
                    fail(BQ_ENOMEM, "server: a request of %llu edges needs %zu bytes, over the budget",
                         (unsigned long long)r->k, bytes);
                    complete_failed(srv, r, BQ_ENOMEM);
                    lk.lock();
                    continue;
                }
                if (srv->inflight.size() + admitted.size() >= srv->cfg.max_inflight ||
                    srv->held_bytes + bytes > budget)
                    break;
                srv->pending.pop_front();
                r->dbytes = bytes;
                srv->held_bytes += bytes;
                admitted.push_back(r);
            }
            idle = admitted.empty() && srv->inflight.empty();
            if (idle) {
                auto drained = [srv] { return srv->to_plan.empty() && srv->planning == 0; };
                if (srv->stop && srv->pending.empty() && drained()) return;
                srv->cv_work.wait(lk, [&] { return !srv->pending.empty() || (srv->stop && drained()); });
                srv->t_idle += lap(t0);
                continue;
            }
        }
        std::vector<Request *> pass, empty;
        for (auto &r : admitted) {
            const int rc = admit(srv, *r);
            if (rc != BQ_OK) {
                complete_failed(srv, r, rc);
                continue;
            }
            pass.push_back(r.get());
            if (r->tasks_total == 0) empty.push_back(r.get());
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->inflight.push_back(r);
        }
        if (!pass.empty()) {
            const int rc = prepare_pass(srv, pass);
            if (rc != BQ_OK) {  // a launch failed: the context is unusable; fail the pass
                for (Request *p : pass) p->status = rc;
            }
        }
        // requests with nothing to count go straight to finalization
        finalize_many(srv, empty);
        const double ta = lap(t0);
        const bool launched = iterate(srv);
        const double tl = lap(t0);
        poll_completions(srv, !launched);
        const double tc = lap(t0);
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->t_admit += ta;
        srv->t_launch += tl;
        srv->t_complete += tc;
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = lo + 1 < v.size() ? lo + 1 : lo;
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace
}  // namespace bq

using namespace bq;

namespace {

void server_free(bq_server *srv) {
    for (int i = 0; i < bq_server::kRing; ++i) {
        if (srv->ring_ev[i]) cudaEventDestroy(srv->ring_ev[i]);
        if (srv->h_items[i]) cudaFreeHost(srv->h_items[i]);
        if (srv->d_items[i]) cudaFree(srv->d_items[i]);
    }
    for (cudaEvent_t e : srv->events) cudaEventDestroy(e);
    srv->events.clear();
    srv->pinned.release();
    if (srv->d_counter) cudaFree(srv->d_counter);
    if (srv->status) cudaFree(srv->status);
    if (srv->stream) cudaStreamDestroy(srv->stream);
    if (srv->copy_stream) cudaStreamDestroy(srv->copy_stream);
    delete srv;
}

}  // namespace

extern "C" {

int bq_server_create(bq_graph *const *graphs, uint32_t n_graphs, const bq_server_config *cfg, bq_server **out) {
    clear_error();
    if (!out) return fail(BQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (!graphs || n_graphs == 0) return fail(BQ_EINVAL, "a server needs at least one graph");
    int dev = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    for (uint32_t i = 0; i < n_graphs; ++i) {
        if (!graphs[i]) return fail(BQ_EINVAL, "graph %u is NULL", i);
        if (graphs[i]->device != dev)
            return fail(BQ_EINVAL, "graph %u lives on device %d, not %d", i, graphs[i]->device, dev);
        if (!graphs[i]->d_rec8) return fail(BQ_EINVAL, "graph %u: the server needs nnz < 2^32", i);
    }
    bq_server_config c{};
    if (cfg) c = *cfg;
    else {
        c.tau_scale = 2.0;
        c.tau_add = 2;
        c.tau_max = 64;
        c.n_scale = 9.0;
        c.n_min = 32;
    }
    if (!c.device_budget_bytes) c.device_budget_bytes = 1ull << 30;
    if (!c.max_inflight) c.max_inflight = 256;
    if (!c.max_pending) c.max_pending = 65536;
    if (!c.tasks_per_iteration) c.tasks_per_iteration = 1ull << 16;
    if (!c.pinned_arena_bytes) c.pinned_arena_bytes = 256ull << 20;
    if (c.max_inflight > (1u << 20)) return fail(BQ_EINVAL, "max_inflight %u is above 2^20", c.max_inflight);
    if (c.tau_max < 1 || !(c.tau_scale >= 0.0) || !(c.n_scale >= 0.0)) return fail(BQ_EINVAL, "bad schedule");
    // the planner reads host copies of the graphs: take them now, before the
    // worker thread exists
    for (uint32_t i = 0; i < n_graphs; ++i) {
        const int rc = graph_fetch_host(graphs[i]);
        if (rc) return rc;
    }
    bq_server *srv = new bq_server();
    srv->graphs.assign(graphs, graphs + n_graphs);
    srv->cfg = c;
    srv->device = dev;
    srv->lanes = tuning_aesc_walks_per_lane();
    cudaError_t e = cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&srv->copy_stream, cudaStreamNonBlocking);
    for (int i = 0; i < bq_server::kRing && e == cudaSuccess; ++i) {
        e = cudaMallocHost((void **)&srv->h_items[i], sizeof(ServeItem) * c.max_inflight);
        if (e == cudaSuccess) e = cudaMalloc((void **)&srv->d_items[i], sizeof(ServeItem) * c.max_inflight);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&srv->ring_ev[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&srv->d_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&srv->status, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(srv->status, 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "bq_server_create");
        server_free(srv);
        return rc;
    }
    {
        // the stream-ordered pool keeps freed request memory (set once per device)
        uint32_t *unused = nullptr;
        int rc = status_word(dev, &unused);
        if (rc == BQ_OK) rc = srv->pinned.reserve(c.pinned_arena_bytes);
        if (rc) {
            server_free(srv);
            return rc;
        }
    }
    srv->t_start = Clock::now();
    uint32_t planners = c.planner_threads;
    if (!planners) {
        const unsigned hw = std::thread::hardware_concurrency();
        planners = std::max(1u, std::min(8u, hw / 2));
    }
    srv->worker = std::thread(worker_main, srv);
    for (uint32_t i = 0; i < planners; ++i) srv->planners.emplace_back(planner_main, srv);
    *out = srv;
    return BQ_OK;
}

int bq_server_submit(bq_server *srv, uint32_t graph, const uint32_t *edges_uv, uint64_t k, double eps,
                     uint64_t seed, uint64_t *request_id) {
    clear_error();
    if (!srv || !request_id) return fail(BQ_EINVAL, "server or request_id is NULL");
    if (graph >= srv->graphs.size()) return fail(BQ_EINVAL, "graph %u of %zu", graph, srv->graphs.size());
    if (k && !edges_uv) return fail(BQ_EINVAL, "edges_uv is NULL");
    if (!(eps > 0.0) || !(eps < 1e6)) return fail(BQ_EINVAL, "eps = %g must be positive", eps);
    if (k >= (1ull << 32)) return fail(BQ_EINVAL, "k = %llu edges in one request", (unsigned long long)k);
    const uint32_t n = srv->graphs[graph]->n;
    for (uint64_t i = 0; i < k; ++i) {
        const uint32_t a = edges_uv[2 * i], b = edges_uv[2 * i + 1];
        if (a >= n || b >= n || a == b)
            return fail(BQ_ENOEDGE, "pair %llu: (%u, %u) is not an edge", (unsigned long long)i, a, b);
    }
    auto r = std::make_shared<Request>();
    r->t_submit = Clock::now();
    r->graph = graph;
    r->k = k;
    r->eps = eps;
    r->seed = seed;
    r->L = layout_of(k);
    r->uv_in.assign(edges_uv, edges_uv + 2 * k);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return fail(BQ_EINVAL, "server is stopping");
        if (srv->to_plan.size() + srv->planning + srv->pending.size() >= srv->cfg.max_pending)
            return fail(BQ_EBUSY, "server queue is full (%u requests)", srv->cfg.max_pending);
        r->id = srv->next_id++;
        srv->to_plan.push_back(r);
        srv->live.insert(r->id);
        ++srv->submitted;
        *request_id = r->id;
    }
    srv->cv_plan.notify_one();
    return BQ_OK;
}

int bq_server_wait(bq_server *srv, uint64_t request_id, double timeout_s, double *sc, uint32_t *counts,
                   double *latency_ms) {
    clear_error();
    if (!srv) return fail(BQ_EINVAL, "server is NULL");
    if (!(timeout_s >= 0.0)) return fail(BQ_EINVAL, "timeout %g", timeout_s);
    RequestPtr r;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        if (!srv->live.count(request_id))
            return fail(BQ_EINVAL, "request %llu is unknown or was already returned", (unsigned long long)request_id);
        const auto deadline =
            Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                               timeout_s > 1e7 ? 1e7 : timeout_s));
        const bool ok = srv->cv_done.wait_until(lk, deadline, [&] { return srv->done.count(request_id) > 0; });
        if (!ok) return fail(BQ_ETIMEOUT, "request %llu is not done", (unsigned long long)request_id);
        auto it = srv->done.find(request_id);
        r = it->second;
        srv->done.erase(it);
        srv->live.erase(request_id);
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (r->status != BQ_OK)
        return fail(r->status, "request %llu: %s", (unsigned long long)request_id,
                    r->error.empty() ? bq_strerror(r->status) : r->error.c_str());
    if (sc && r->k) memcpy(sc, r->h_out + (r->L.sc - r->L.out), 8 * r->k);
    if (counts && r->k) memcpy(counts, r->h_out + (r->L.counts - r->L.out), 16 * r->k);
    srv->pinned.put(r->h_out, r->h_out_cap);
    r->h_out = nullptr;
    return BQ_OK;
}

int bq_server_stats_get(bq_server *srv, bq_server_stats *out) {
    clear_error();
    if (!srv || !out) return fail(BQ_EINVAL, "server or out is NULL");
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        out->submitted = srv->submitted;
        out->completed = srv->completed;
        out->failed = srv->failed;
        out->edges_completed = srv->edges_completed;
        out->iterations = srv->iterations;
        out->walk_steps = srv->walk_steps;
        out->inflight = (uint32_t)srv->inflight.size();
        out->pending = (uint32_t)(srv->to_plan.size() + srv->planning + srv->pending.size());
        out->worker_admit_s = srv->t_admit;
        out->worker_launch_s = srv->t_launch;
        out->worker_complete_s = srv->t_complete;
        out->worker_idle_s = srv->t_idle;
        out->planner_s = srv->t_plan;
        out->planner_max_ms = srv->t_plan_max * 1e3;
        {
            std::lock_guard<std::mutex> plk(srv->pinned.mu);
            out->pinned_fallbacks = srv->pinned.fallbacks;
            out->pinned_fallback_s = srv->pinned.fallback_s;
        }
        lat = srv->latencies_ms;
    }
    out->p50_ms = percentile(lat, 0.50);
    out->p99_ms = percentile(lat, 0.99);
    out->uptime_s = std::chrono::duration<double>(Clock::now() - srv->t_start).count();
    return BQ_OK;
}

int bq_server_destroy(bq_server *srv) {
    clear_error();
    if (!srv) return BQ_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_plan.notify_all();
    srv->cv_work.notify_all();
    for (auto &t : srv->planners)
        if (t.joinable()) t.join();
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    cudaStreamSynchronize(srv->stream);
    cudaStreamSynchronize(srv->copy_stream);
    server_free(srv);
    cudaSetDevice(prev);
    return BQ_OK;
}

}  // extern "C"
