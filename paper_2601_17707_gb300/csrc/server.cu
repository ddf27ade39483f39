// server.cu -- the serving loop of include/bbc.h (bbc_server_*, bbc_submit, bbc_poll,
// bbc_wait): continuous batching of many graph-counting requests on one GPU.
//
// Requests are copied at submit time and queued. Then:
//   1. admission: queued requests are admitted in arrival order while the device memory
//      reserved for admitted requests plus theirs stays within the budget;
//   2. a pool of preparation threads, each on its own stream, prepares admitted requests
//      (bbc_prepare's pipeline) and zeroes their counts; their device layout stays
//      resident until done;
// and a tick thread repeats:
//   3. one launch of the counting kernels covers every prepared graph: all remaining work
//      items of the small ones and a bounded chunk of each large one, so a large request
//      advances over several ticks (its partial totals stay in device memory between
//      ticks) and never holds small requests back for long;
//   4. requests whose work items are all counted complete: their totals are read back,
//      their device memory is freed and the reservation released.
// Requests that arrive while a tick runs join at the next tick: the GPU work of all
// admitted requests overlaps inside each tick's launch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "graph.cuh"

namespace bbc {
namespace {

using Clock = std::chrono::steady_clock;
// Preparation threads per server. Preparing a small request is mostly kernel launches
// and stream synchronisations, which contend in the driver: 16 threads prepared fewer
// requests per second than 6 (2,390 against 2,720 at saturation).
constexpr int kPrepThreads = 6;

struct Request {
    uint64_t ticket = 0;
    int32_t n_u = 0, n_v = 0;
    int64_t n_edges = 0;
    std::vector<int32_t> u, v;
    std::vector<int8_t> s;
    size_t reserve = 0;          // device bytes reserved at admission
    bbc_graph *g = nullptr;
    int32_t tile_done = 0, warp_done = 0, wt_done = 0, gt_done = 0;
    bool done = false;
    bool waited = false;         // found the budget full at submission
    bbc_status status = BBC_OK;
    uint64_t balanced = 0;
    uint64_t wedges = 0;         // W of the prepared graph
    int32_t ticks = 0;           // counting launches this request took part in
    double gpu_us = 0;           // device time of those launches (shared with the others)
    Clock::time_point t_submit, t_admit, t_ready, t_done;
};

// Device memory a request may hold at its peak (preparation temporaries included).
size_t reservation_bytes(int32_t n_u, int32_t n_v, int64_t n_edges) {
    return (size_t)n_edges * 56 + ((size_t)n_u + (size_t)n_v) * 48 + (size_t(1) << 20);
}

template <class T>
bbc_status ensure(T **buf, size_t *cap, size_t need, cudaStream_t st) {
    if (*cap >= need && *buf) return BBC_OK;
    if (*buf) dev_free(*buf, st);
    *buf = nullptr;
    size_t n = std::max(need, *cap * 2);
    BBC_TRY(dev_alloc_n(buf, n, st));
    *cap = n;
    return BBC_OK;
}

}  // namespace
}  // namespace bbc

struct bbc_server {
    size_t budget = 0;
    bbc::Tuning tuning{};
    int device = 0;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_prep;
    std::deque<bbc::Request *> queue;      // submitted, not admitted
    std::deque<bbc::Request *> to_prepare; // admitted
    std::vector<bbc::Request *> ready;     // prepared, not yet counting
    int preparing = 0;
    std::vector<std::thread> preppers;
    std::vector<bbc::Request *> active;
    std::unordered_map<uint64_t, bbc::Request *> all;
    size_t reserved = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::vector<double> latencies_us;
    // counters (bbc_server_counters_get)
    std::chrono::steady_clock::time_point t_created;
    uint64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_waited = 0;
    uint64_t n_ticks = 0, max_queue = 0, max_resident = 0;
    double tick_wall_us = 0, tick_gpu_us = 0, prep_wall_us = 0;
    size_t peak_reserved = 0;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    // tick buffers (grown as needed)
    bbc::DevGraph *dgraphs = nullptr;
    size_t dgraphs_cap = 0;
    bbc::TileItem *tiles = nullptr;
    size_t tiles_cap = 0;
    bbc::HashItem *warps = nullptr;
    size_t warps_cap = 0;
    bbc::HashItem *wts = nullptr;
    size_t wts_cap = 0;
    bbc::HashItem *gts = nullptr;
    size_t gts_cap = 0;
    bbc::CopyJob *djobs = nullptr;
    size_t djobs_cap = 0;
    bbc::QueueState *queue_state = nullptr;
    unsigned long long *host_totals = nullptr;  // pinned, 2 per active request
    size_t host_totals_cap = 0;
};

namespace bbc {
namespace {

void finish_locked(bbc_server *S, Request *r, bbc_status st, uint64_t balanced) {
    r->status = st;
    r->balanced = balanced;
    r->done = true;
    r->t_done = Clock::now();
    S->n_completed++;
    r->u = {};
    r->v = {};
    r->s = {};
    if (st == BBC_OK)
        S->latencies_us.push_back(
            std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
}

// Moves queued requests to the preparation queue while their reservations fit.
void admit_locked(bbc_server *S) {
    bool any = false;
    while (!S->queue.empty() && S->reserved + S->queue.front()->reserve <= S->budget) {
        Request *r = S->queue.front();
        S->queue.pop_front();
        S->reserved += r->reserve;
        S->peak_reserved = std::max(S->peak_reserved, S->reserved);
        S->n_admitted++;
        if (r->waited) S->n_waited++;
        r->t_admit = Clock::now();
        S->to_prepare.push_back(r);
        any = true;
    }
    if (!S->queue.empty()) {
        // whoever is still queued now waits for memory to be released
        for (Request *q : S->queue) q->waited = true;
    }
    const uint64_t resident = (uint64_t)(S->to_prepare.size() + S->ready.size() + S->active.size()) +
                              (uint64_t)S->preparing;
    S->max_resident = std::max(S->max_resident, resident);
    if (any) S->cv_prep.notify_all();
}

// A preparation thread: prepares admitted requests on its own stream, waits for that
// stream, and hands the graph to the tick thread. A failed request completes with its
// status and releases its reservation.
void prep_main(bbc_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_prep.wait(lk, [&] { return S->stop || !S->to_prepare.empty(); });
            if (S->stop) break;
            r = S->to_prepare.front();
            S->to_prepare.pop_front();
            S->preparing++;
        }
        const Clock::time_point t0 = Clock::now();
        bbc_graph *g = nullptr;
        bbc_status s = prepare_graph(r->n_u, r->n_v, r->n_edges, r->u.data(), r->v.data(),
                                     r->s.data(), 0u, st, &g);
        if (s == BBC_OK) s = build_work_lists(g, S->tuning, st);
        // centre-split parts of one tile may run in different ticks: their merged
        // counters are cleared once, here
        if (s == BBC_OK) s = clear_centre_split(g, st);
        if (s == BBC_OK) {
            cudaError_t e = cudaMemsetAsync(g->totals, 0, 16, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_fail(e, "server preparation");
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->preparing--;
        r->t_ready = Clock::now();
        S->prep_wall_us += std::chrono::duration<double, std::micro>(r->t_ready - t0).count();
        if (s != BBC_OK) {
            if (g) release_graph(g, st);
            S->reserved -= r->reserve;
            finish_locked(S, r, s, 0);
            admit_locked(S);
            S->cv_done.notify_all();
        } else {
            r->g = g;
            r->wedges = g->wedges;
            r->u = {};
            r->v = {};
            r->s = {};
            S->ready.push_back(r);
            S->cv_work.notify_one();
        }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
}

// One tick over the active requests: a combined work list and one counting launch.
bbc_status run_tick(bbc_server *S, std::vector<Request *> &act) {
    cudaStream_t st = S->stream;
    const int chunk = 4 * device_sm_count() * S->tuning.blocks_per_sm;
    const size_t n = act.size();
    std::vector<DevGraph> hd(n);
    std::vector<CopyJob> jt, jh, jw, jg;
    int64_t nt = 0, nh = 0, nw = 0, ngr = 0;
    std::vector<int32_t> take_t(n), take_h(n), take_w(n), take_g(n);
    for (size_t i = 0; i < n; ++i) {
        bbc_graph *g = act[i]->g;
        hd[i] = host_descriptor(g, false, true);
        const int32_t rt = g->n_tile - act[i]->tile_done;
        const int32_t rh = g->n_warp - act[i]->warp_done;
        const int32_t rw = g->n_wt - act[i]->wt_done;
        const int32_t rg = g->n_gt - act[i]->gt_done;
        take_t[i] = std::min(rt, chunk);
        take_h[i] = std::min(rh, 64 * chunk);
        take_w[i] = std::min(rw, 16 * chunk);
        take_g[i] = std::min(rg, 4 * chunk);
        if (take_t[i] > 0)
            jt.push_back(CopyJob{g->tile_items + act[i]->tile_done, nt, take_t[i], (int32_t)i});
        if (take_h[i] > 0)
            jh.push_back(CopyJob{g->warp_items + act[i]->warp_done, nh, take_h[i], (int32_t)i});
        if (take_w[i] > 0)
            jw.push_back(CopyJob{g->wt_items + act[i]->wt_done, nw, take_w[i], (int32_t)i});
        if (take_g[i] > 0)
            jg.push_back(CopyJob{g->gt_items + act[i]->gt_done, ngr, take_g[i], (int32_t)i});
        nt += take_t[i];
        nh += take_h[i];
        nw += take_w[i];
        ngr += take_g[i];
    }
    BBC_TRY(ensure(&S->dgraphs, &S->dgraphs_cap, n, st));
    BBC_TRY(ensure(&S->tiles, &S->tiles_cap, (size_t)std::max<int64_t>(nt, 1), st));
    BBC_TRY(ensure(&S->warps, &S->warps_cap, (size_t)std::max<int64_t>(nh, 1), st));
    BBC_TRY(ensure(&S->wts, &S->wts_cap, (size_t)std::max<int64_t>(nw, 1), st));
    BBC_TRY(ensure(&S->gts, &S->gts_cap, (size_t)std::max<int64_t>(ngr, 1), st));
    BBC_TRY(ensure(&S->djobs, &S->djobs_cap,
                   std::max(std::max(jt.size(), jg.size()), std::max(jh.size(), jw.size())) + 1, st));
    if (!S->queue_state) BBC_TRY(dev_alloc_n(&S->queue_state, 1, st));
    if (S->host_totals_cap < 2 * n) {
        if (S->host_totals) cudaFreeHost(S->host_totals);
        S->host_totals = nullptr;
        S->host_totals_cap = std::max<size_t>(2 * n, 2 * S->host_totals_cap);
        BBC_CUDA_TRY(cudaMallocHost(&S->host_totals, sizeof(unsigned long long) * S->host_totals_cap));
    }
    BBC_CUDA_TRY(cudaMemcpyAsync(S->dgraphs, hd.data(), sizeof(DevGraph) * n, cudaMemcpyHostToDevice, st));
    BBC_TRY(concat_items(jt, true, S->tiles, S->djobs, st));
    BBC_TRY(concat_items(jh, false, S->warps, S->djobs, st));
    BBC_TRY(concat_items(jw, false, S->wts, S->djobs, st));
    BBC_TRY(concat_items(jg, false, S->gts, S->djobs, st));
    BBC_CUDA_TRY(cudaMemsetAsync(S->queue_state, 0, sizeof(QueueState), st));
    CountLaunch L{};
    L.graphs = S->dgraphs;
    L.tile_items = S->tiles;
    L.n_tile_items = (int32_t)nt;
    L.warp_items = S->warps;
    L.n_warp_items = (int32_t)nh;
    L.wt_items = S->wts;
    L.n_wt_items = (int32_t)nw;
    L.gt_items = S->gts;
    L.n_gt_items = (int32_t)ngr;
    L.queue = S->queue_state;
    L.tuning = S->tuning;
    for (size_t i = 0; i < n; ++i) L.prefetch = L.prefetch || rows_exceed_l2(act[i]->g);
    BBC_CUDA_TRY(cudaEventRecord(S->ev_a, st));
    BBC_TRY(launch_count(L, st));
    BBC_CUDA_TRY(cudaEventRecord(S->ev_b, st));
    for (size_t i = 0; i < n; ++i) {
        act[i]->tile_done += take_t[i];
        act[i]->warp_done += take_h[i];
        act[i]->wt_done += take_w[i];
        act[i]->gt_done += take_g[i];
        BBC_CUDA_TRY(cudaMemcpyAsync(S->host_totals + 2 * i, act[i]->g->totals, 16,
                                     cudaMemcpyDeviceToHost, st));
    }
    QueueState qs{};
    BBC_CUDA_TRY(cudaMemcpyAsync(&qs, S->queue_state, sizeof qs, cudaMemcpyDeviceToHost, st));
    BBC_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    BBC_CUDA_TRY(cudaEventElapsedTime(&ms, S->ev_a, S->ev_b));
    for (size_t i = 0; i < n; ++i) {
        act[i]->ticks++;
        act[i]->gpu_us += 1e3 * (double)ms;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->n_ticks++;
        S->tick_gpu_us += 1e3 * (double)ms;
    }
    if (qs.error) {
        set_error("serving tick: counting kernel reported an internal inconsistency");
        return BBC_E_CUDA;
    }
    return BBC_OK;
}

void worker_main(bbc_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request *> act;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->ready.empty() || !S->active.empty(); });
            if (S->stop) break;
            for (Request *r : S->ready) S->active.push_back(r);
            S->ready.clear();
            act = S->active;
        }
        if (act.empty()) continue;
        const Clock::time_point t0 = Clock::now();
        const bbc_status st = run_tick(S, act);
        std::lock_guard<std::mutex> lk(S->mu);
        S->tick_wall_us += std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
        std::vector<Request *> still;
        for (size_t i = 0; i < act.size(); ++i) {
            Request *r = act[i];
            const bool complete = r->tile_done >= r->g->n_tile && r->warp_done >= r->g->n_warp &&
                                  r->wt_done >= r->g->n_wt && r->gt_done >= r->g->n_gt;
            if (st != BBC_OK || complete) {
                release_graph(r->g, S->stream);
                r->g = nullptr;
                S->reserved -= r->reserve;
                finish_locked(S, r, st, st == BBC_OK ? S->host_totals[2 * i] : 0);
            } else {
                still.push_back(r);
            }
        }
        S->active = still;
        admit_locked(S);
        S->cv_done.notify_all();
    }
}

}  // namespace
}  // namespace bbc

using namespace bbc;

extern "C" {

bbc_status bbc_server_create(size_t device_budget_bytes, const bbc_tuning *tuning, bbc_server **out) {
    if (!out || device_budget_bytes == 0) {
        set_error("bbc_server_create: NULL output or zero budget");
        return BBC_E_INVALID_ARG;
    }
    try {
        bbc_server *S = new bbc_server();
        S->budget = device_budget_bytes;
        S->tuning = resolve_tuning(tuning, device_sm_count());
        if (S->tuning.split_wedges == 0) S->tuning.split_wedges = (long long)1 << 26;
        cudaGetDevice(&S->device);
        S->t_created = Clock::now();
        cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&S->ev_a);
        if (e == cudaSuccess) e = cudaEventCreate(&S->ev_b);
        if (e != cudaSuccess) {
            if (S->ev_a) cudaEventDestroy(S->ev_a);
            if (S->stream) cudaStreamDestroy(S->stream);
            delete S;
            return cuda_fail(e, "bbc_server_create stream");
        }
        S->worker = std::thread(worker_main, S);
        for (int i = 0; i < kPrepThreads; ++i) S->preppers.emplace_back(prep_main, S);
        *out = S;
        return BBC_OK;
    } catch (...) {
        set_error("bbc_server_create failed");
        return BBC_E_NO_MEMORY;
    }
}

bbc_status bbc_submit(bbc_server *S, int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *u,
                      const int32_t *v, const int8_t *sign, uint64_t *ticket) {
    if (!S || !ticket || n_u < 0 || n_v < 0 || n_edges < 0 || (n_edges > 0 && (!u || !v || !sign))) {
        set_error("bbc_submit: bad arguments");
        return BBC_E_INVALID_ARG;
    }
    const size_t need = reservation_bytes(n_u, n_v, n_edges);
    if (need > S->budget) {
        set_error("bbc_submit: the request alone needs more device memory than the budget");
        return BBC_E_OVER_BUDGET;
    }
    try {
        Request *r = new Request();
        r->n_u = n_u;
        r->n_v = n_v;
        r->n_edges = n_edges;
        r->u.assign(u, u + n_edges);
        r->v.assign(v, v + n_edges);
        r->s.assign(sign, sign + n_edges);
        r->reserve = need;
        r->t_submit = Clock::now();
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return BBC_E_CANCELLED;
        }
        r->ticket = S->next_ticket++;
        S->all[r->ticket] = r;
        S->queue.push_back(r);
        S->n_submitted++;
        *ticket = r->ticket;
        admit_locked(S);
        S->max_queue = std::max<uint64_t>(S->max_queue, S->queue.size());
        return BBC_OK;
    } catch (...) {
        set_error("bbc_submit: host allocation failed");
        return BBC_E_NO_MEMORY;
    }
}

bbc_status bbc_poll(bbc_server *S, uint64_t ticket, uint64_t *balanced) {
    if (!S) return BBC_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) {
        set_error("bbc_poll: unknown ticket");
        return BBC_E_INVALID_ARG;
    }
    Request *r = it->second;
    if (!r->done) return BBC_E_NOT_READY;
    if (balanced && r->status == BBC_OK) *balanced = r->balanced;
    return r->status;
}

bbc_status bbc_wait(bbc_server *S, uint64_t ticket, int64_t timeout_us, uint64_t *balanced) {
    if (!S) return BBC_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) {
        set_error("bbc_wait: unknown ticket");
        return BBC_E_INVALID_ARG;
    }
    Request *r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_us < 0)
        S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
        return BBC_E_TIMEOUT;
    if (balanced && r->status == BBC_OK) *balanced = r->balanced;
    return r->status;
}

bbc_status bbc_server_stats(bbc_server *S, uint64_t *completed, double *p50_us, double *p99_us,
                            double *mean_us) {
    if (!S) return BBC_E_INVALID_ARG;
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        lat = S->latencies_us;
    }
    if (completed) *completed = lat.size();
    double p50 = 0, p99 = 0, mean = 0;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double q) {
            const size_t k = std::min(lat.size() - 1, (size_t)(q * (double)(lat.size() - 1) + 0.5));
            return lat[k];
        };
        p50 = pct(0.50);
        p99 = pct(0.99);
        for (double x : lat) mean += x;
        mean /= (double)lat.size();
    }
    if (p50_us) *p50_us = p50;
    if (p99_us) *p99_us = p99;
    if (mean_us) *mean_us = mean;
    return BBC_OK;
}

bbc_status bbc_server_counters_get(bbc_server *S, bbc_server_counters *out) {
    if (!S || !out) {
        set_error("bbc_server_counters_get: NULL argument");
        return BBC_E_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    bbc_server_counters c{};
    c.submitted = S->n_submitted;
    c.admitted = S->n_admitted;
    c.completed = S->n_completed;
    c.admitted_after_wait = S->n_waited;
    c.queued_now = S->queue.size();
    c.max_queued = S->max_queue;
    c.max_resident = S->max_resident;
    c.ticks = S->n_ticks;
    c.budget_bytes = S->budget;
    c.reserved_bytes = S->reserved;
    c.peak_reserved_bytes = S->peak_reserved;
    c.tick_wall_us = S->tick_wall_us;
    c.tick_gpu_us = S->tick_gpu_us;
    c.prep_wall_us = S->prep_wall_us;
    c.elapsed_us = std::chrono::duration<double, std::micro>(Clock::now() - S->t_created).count();
    *out = c;
    return BBC_OK;
}

bbc_status bbc_server_request_info(bbc_server *S, uint64_t ticket, bbc_request_info *out) {
    if (!S || !out) {
        set_error("bbc_server_request_info: NULL argument");
        return BBC_E_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) {
        set_error("bbc_server_request_info: unknown ticket");
        return BBC_E_INVALID_ARG;
    }
    const Request *r = it->second;
    if (!r->done) return BBC_E_NOT_READY;
    auto us = [](Clock::time_point a, Clock::time_point b) {
        return std::chrono::duration<double, std::micro>(b - a).count();
    };
    bbc_request_info q{};
    q.status = r->status;
    q.n_edges = r->n_edges;
    q.wedges = r->wedges;
    q.reserved_bytes = r->reserve;
    q.ticks = r->ticks;
    q.waited_for_memory = r->waited ? 1 : 0;
    const bool admitted = r->t_admit.time_since_epoch().count() != 0;
    const bool prepared = r->t_ready.time_since_epoch().count() != 0;
    q.latency_us = us(r->t_submit, r->t_done);
    q.queued_us = admitted ? us(r->t_submit, r->t_admit) : q.latency_us;
    q.prepare_us = admitted && prepared ? us(r->t_admit, r->t_ready) : 0.0;
    q.count_us = prepared ? us(r->t_ready, r->t_done) : 0.0;
    q.tick_gpu_us = r->gpu_us;
    q.submit_us = us(S->t_created, r->t_submit);
    *out = q;
    return BBC_OK;
}

void bbc_server_destroy(bbc_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Request *r : S->queue) finish_locked(S, r, BBC_E_CANCELLED, 0);
        S->queue.clear();
        for (Request *r : S->to_prepare) finish_locked(S, r, BBC_E_CANCELLED, 0);
        S->to_prepare.clear();
        S->cv_work.notify_all();
        S->cv_prep.notify_all();
        S->cv_done.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (std::thread &t : S->preppers)
        if (t.joinable()) t.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (Request *r : S->ready) {
        if (r->g) release_graph(r->g, S->stream);
        r->g = nullptr;
        finish_locked(S, r, BBC_E_CANCELLED, 0);
    }
    for (Request *r : S->active) {
        if (r->g) release_graph(r->g, S->stream);
        r->g = nullptr;
        if (!r->done) finish_locked(S, r, BBC_E_CANCELLED, 0);
    }
    void *bufs[] = {S->dgraphs, S->tiles, S->warps, S->wts, S->gts, S->djobs, S->queue_state};
    for (void *p : bufs)
        if (p) dev_free(p, S->stream);
    cudaStreamSynchronize(S->stream);
    if (S->host_totals) cudaFreeHost(S->host_totals);
    cudaEventDestroy(S->ev_a);
    cudaEventDestroy(S->ev_b);
    cudaStreamDestroy(S->stream);
    cudaSetDevice(prev);
    for (auto &kv : S->all) delete kv.second;
    delete S;
}

}  // extern "C"
