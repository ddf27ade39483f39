// batch.cu -- bbc_count_batch / bbc_autotune_batch: many prepared graphs counted by one
// persistent launch over a device-side (graph, anchor, tile range) work list.
//
// A "plan" concatenates the member graphs' work items (tagging each with its graph
// index) graph by graph, heaviest graph first, and records the memsets and counting
// launches into a CUDA graph once. Later
// calls with the same graphs and tuning replay that graph: one launch of the whole
// counting step, whatever the number of graphs.
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "graph.cuh"

namespace bbc {
namespace {

constexpr int kThreads = 256;

template <class Item>
__global__ void k_concat_items(const CopyJob *__restrict__ jobs, Item *__restrict__ dst) {
    const CopyJob j = jobs[blockIdx.x];
    const Item *src = static_cast<const Item *>(j.src);
    for (int i = threadIdx.x; i < j.n; i += blockDim.x) {
        Item it = src[i];
        it.graph = j.graph;
        dst[j.dst + i] = it;
    }
}

struct Plan {
    std::vector<uint64_t> uids;
    std::vector<uint64_t> versions;   // each graph's layout_version when the plan was built
    Tuning tuning{};
    int device = 0;
    int32_t n = 0;
    DevGraph *dgraphs = nullptr;
    unsigned long long *totals = nullptr;     // 2 per graph
    unsigned long long *host_totals = nullptr;  // pinned: 2 per graph, then the error word
    QueueState *queue = nullptr;
    TileItem *tiles = nullptr;
    HashItem *warp = nullptr;
    HashItem *wt = nullptr;
    HashItem *gt = nullptr;
    int32_t n_tile = 0, n_warp = 0, n_wt = 0, n_gt = 0;
    cudaStream_t stream = nullptr;            // capture / replay stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    CountLaunch launch{};                     // what the graph records (for profiled runs)
    std::vector<const bbc_graph *> cs_graphs; // members with centre-split tiles (cleared per run)

    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        void *ps[] = {dgraphs, totals, queue, tiles, warp, wt, gt};
        for (void *p : ps)
            if (p) dev_free(p, stream);
        if (stream) cudaStreamSynchronize(stream);
        if (host_totals) cudaFreeHost(host_totals);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (stream) cudaStreamDestroy(stream);
    }
};

// The queue's error word, copied back after the totals of each replay.
unsigned *host_error_word(Plan *p) { return reinterpret_cast<unsigned *>(p->host_totals + 2 * (size_t)p->n); }

std::mutex g_plan_mu;
std::vector<std::unique_ptr<Plan>> g_plans;  // most recent last; a handful kept
constexpr size_t kMaxPlans = 4;

std::mutex g_tune_mu;
std::map<std::vector<long long>, Tuning> g_tuned;
bool g_tune_loaded = false;

// The persisted tuning cache: one line per shape key, "key... : tile_words warp_max_wedges
// split_wedges blocks_per_sm queue_chunk group_warps". Its path is $BBC_TUNE_CACHE, else
// $XDG_CACHE_HOME/bbc/batch_tuning.txt, else $HOME/.cache/bbc/batch_tuning.txt; an empty
// BBC_TUNE_CACHE turns persistence off.
std::string tune_cache_path() {
    if (const char *p = getenv("BBC_TUNE_CACHE")) return std::string(p);
    if (const char *x = getenv("XDG_CACHE_HOME"); x && *x) return std::string(x) + "/bbc/batch_tuning.txt";
    if (const char *h = getenv("HOME"); h && *h) return std::string(h) + "/.cache/bbc/batch_tuning.txt";
    return std::string();
}

void load_tune_cache_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        std::vector<long long> key;
        char *colon = strchr(line, ':');
        if (!colon) continue;
        *colon = 0;
        char *p = line, *end = nullptr;
        for (;;) {
            const long long v = strtoll(p, &end, 10);
            if (end == p) break;
            key.push_back(v);
            p = end;
        }
        long long tw = 0, wm = 0, sp = 0, bp = 0, qc = 0, gw = 0;
        if (key.size() != 5 ||
            sscanf(colon + 1, "%lld %lld %lld %lld %lld %lld", &tw, &wm, &sp, &bp, &qc, &gw) != 6)
            continue;
        bbc_tuning t{};
        t.tile_words = (int32_t)tw;
        t.warp_max_wedges = (int32_t)wm;
        t.split_wedges = (int32_t)std::min<long long>(sp, INT32_MAX);
        t.blocks_per_sm = (int32_t)bp;
        t.queue_chunk = (int32_t)qc;
        t.group_warps = (int32_t)gw;
        g_tuned[key] = resolve_tuning(&t, device_sm_count());
    }
    fclose(f);
}

// Rewrites the cache file with every tuned entry of this process (best effort: a cache
// that cannot be written only costs a new search next time).
void save_tune_cache_locked() {
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        // create the directory chain (mkdir -p)
        for (size_t i = 1; i <= slash; ++i)
            if (path[i] == '/' || i == slash) mkdir(path.substr(0, i == slash ? slash : i).c_str(), 0755);
    }
    const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const auto &kv : g_tuned) {
        for (long long v : kv.first) fprintf(f, "%lld ", v);
        const Tuning &t = kv.second;
        fprintf(f, ": %d %d %lld %d %d %d\n", t.tile_words, t.warp_max_wedges, t.split_wedges,
                t.blocks_per_sm, t.queue_chunk, t.group_warps);
    }
    const bool ok = fclose(f) == 0;
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
}

std::vector<long long> shape_key(int32_t n, bbc_graph *const *gs) {
    long long e = 0, w = 0, s = 0;
    for (int i = 0; i < n; ++i) {
        e += gs[i]->n_edges;
        w += (long long)gs[i]->wedges;
        s += gs[i]->nS;
    }
    // coarse buckets (powers of two) so similar batches share a tuned choice
    auto bucket = [](long long x) {
        int b = 0;
        while (x > 1) {
            x >>= 1;
            ++b;
        }
        return (long long)b;
    };
    return {device_sm_count(), n, bucket(e), bucket(w), bucket(s)};
}

bool same_tuning(const Tuning &a, const Tuning &b) {
    return a.tile_words == b.tile_words && a.warp_max_wedges == b.warp_max_wedges &&
           a.split_wedges == b.split_wedges && a.blocks_per_sm == b.blocks_per_sm &&
           a.plain == b.plain && a.queue_chunk == b.queue_chunk && a.group_warps == b.group_warps;
}

#define BBC_LAUNCH_OK(what)                                        \
    do {                                                           \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return ::bbc::cuda_fail(_e, what);  \
    } while (0)

bbc_status build_plan(int32_t n, bbc_graph *const *gs, const Tuning &T, std::unique_ptr<Plan> &out) {
    auto P = std::make_unique<Plan>();
    P->n = n;
    P->tuning = T;
    cudaGetDevice(&P->device);
    BBC_CUDA_TRY(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    BBC_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
    BBC_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
    cudaStream_t st = P->stream;
    for (int i = 0; i < n; ++i) {
        P->uids.push_back(gs[i]->uid);
        if (gs[i]->device != P->device) {
            set_error("bbc_count_batch: graphs prepared on another device");
            return BBC_E_INVALID_ARG;
        }
        BBC_TRY(build_work_lists(gs[i], T, st));
        P->versions.push_back(gs[i]->layout_version);
    }
    std::vector<DevGraph> hd(n);
    std::vector<CopyJob> jt, jh, jw, jg;
    int64_t nt = 0, nh = 0, nw = 0, ngr = 0;
    BBC_TRY(dev_alloc_n(&P->totals, (size_t)2 * n, st));
    for (int i = 0; i < n; ++i) {
        hd[i] = host_descriptor(gs[i], false, true);
        hd[i].totals = P->totals + 2 * i;
    }
    // Graph-major queues, heaviest graph first: a graph's items stay together, so only a
    // few graphs' rows are being read at any time and they stay in L2.
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return gs[x]->wedges > gs[y]->wedges; });
    for (int i : order) {
        bbc_graph *g = gs[i];
        if (g->n_tile) jt.push_back(CopyJob{g->tile_items, nt, g->n_tile, i});
        if (g->n_warp) jh.push_back(CopyJob{g->warp_items, nh, g->n_warp, i});
        if (g->n_wt) jw.push_back(CopyJob{g->wt_items, nw, g->n_wt, i});
        if (g->n_gt) jg.push_back(CopyJob{g->gt_items, ngr, g->n_gt, i});
        nt += g->n_tile;
        nh += g->n_warp;
        nw += g->n_wt;
        ngr += g->n_gt;
    }
    if (nt > INT32_MAX || nh > INT32_MAX || nw > INT32_MAX || ngr > INT32_MAX) {
        set_error("bbc_count_batch: too many work items");
        return BBC_E_INVALID_ARG;
    }
    P->n_tile = (int32_t)nt;
    P->n_warp = (int32_t)nh;
    P->n_wt = (int32_t)nw;
    P->n_gt = (int32_t)ngr;
    BBC_TRY(dev_alloc_n(&P->dgraphs, (size_t)n, st));
    BBC_TRY(dev_alloc_n(&P->queue, 1, st));
    BBC_TRY(dev_alloc_n(&P->tiles, (size_t)nt, st));
    BBC_TRY(dev_alloc_n(&P->warp, (size_t)nh, st));
    BBC_TRY(dev_alloc_n(&P->wt, (size_t)nw, st));
    BBC_TRY(dev_alloc_n(&P->gt, (size_t)ngr, st));
    BBC_CUDA_TRY(cudaMallocHost(&P->host_totals, sizeof(unsigned long long) * (2 * (size_t)n + 1)));
    memset(P->host_totals, 0, sizeof(unsigned long long) * (2 * (size_t)n + 1));
    BBC_CUDA_TRY(cudaMemcpyAsync(P->dgraphs, hd.data(), sizeof(DevGraph) * (size_t)n,
                                 cudaMemcpyHostToDevice, st));
    // concatenate, tagging each item with its graph index
    CopyJob *djobs = nullptr;
    const size_t maxj = std::max(std::max(jt.size(), jg.size()), std::max(jh.size(), jw.size()));
    BBC_TRY(dev_alloc_n(&djobs, maxj, st));
    struct Part {
        std::vector<CopyJob> *jobs;
        int which;
    } parts[4] = {{&jt, 0}, {&jh, 2}, {&jw, 3}, {&jg, 4}};
    bbc_status s = BBC_OK;
    for (auto &pt : parts) {
        if (pt.jobs->empty()) continue;
        cudaError_t e = cudaMemcpyAsync(djobs, pt.jobs->data(), sizeof(CopyJob) * pt.jobs->size(),
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            s = cuda_fail(e, "batch job copy");
            break;
        }
        const unsigned nb = (unsigned)pt.jobs->size();
        note_launch();
        if (pt.which == 0) k_concat_items<TileItem><<<nb, kThreads, 0, st>>>(djobs, P->tiles);
        if (pt.which == 2) k_concat_items<HashItem><<<nb, kThreads, 0, st>>>(djobs, P->warp);
        if (pt.which == 3) k_concat_items<HashItem><<<nb, kThreads, 0, st>>>(djobs, P->wt);
        if (pt.which == 4) k_concat_items<HashItem><<<nb, kThreads, 0, st>>>(djobs, P->gt);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // djobs is reused
        if (e != cudaSuccess) {
            s = cuda_fail(e, "k_concat_items");
            break;
        }
    }
    dev_free(djobs, st);
    BBC_TRY(s);
    BBC_CUDA_TRY(cudaStreamSynchronize(st));
    // record the counting step once
    BBC_TRY(configure_count_kernels());
    CountLaunch L{};
    L.graphs = P->dgraphs;
    L.tile_items = P->tiles;
    L.n_tile_items = P->n_tile;
    L.warp_items = P->warp;
    L.n_warp_items = P->n_warp;
    L.wt_items = P->wt;
    L.n_wt_items = P->n_wt;
    L.gt_items = P->gt;
    L.n_gt_items = P->n_gt;
    L.queue = P->queue;
    L.tuning = T;
    for (int i = 0; i < n; ++i) L.prefetch = L.prefetch || rows_exceed_l2(gs[i]);
    P->launch = L;
    for (int i = 0; i < n; ++i)
        if (gs[i]->n_cs_groups > 0) P->cs_graphs.push_back(gs[i]);
    BBC_TRY(configure_count_kernels());
    BBC_TRY(ensure_side_streams());   // no stream or event creation inside the capture
    BBC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(P->totals, 0, sizeof(unsigned long long) * 2 * (size_t)n, st);
    cudaMemsetAsync(P->queue, 0, sizeof(QueueState), st);
    bbc_status ls = BBC_OK;
    for (const bbc_graph *cg : P->cs_graphs)
        if (ls == BBC_OK) ls = clear_centre_split(cg, st);
    if (ls == BBC_OK) ls = launch_count(L, st);
    cudaMemcpyAsync(P->host_totals, P->totals, sizeof(unsigned long long) * 2 * (size_t)n,
                    cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(host_error_word(P.get()), &P->queue->error, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    BBC_TRY(ls);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&P->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    out = std::move(P);
    return BBC_OK;
}

Plan *find_or_build(int32_t n, bbc_graph *const *gs, const Tuning &T, bbc_status *status) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    for (size_t k = 0; k < g_plans.size(); ++k) {
        Plan *p = g_plans[k].get();
        if (p->n != n || p->device != dev || !same_tuning(p->tuning, T)) continue;
        bool same = true;
        for (int i = 0; i < n && same; ++i)
            same = p->uids[i] == gs[i]->uid && p->versions[i] == gs[i]->layout_version;
        if (same) {
            auto keep = std::move(g_plans[k]);
            g_plans.erase(g_plans.begin() + (long)k);
            g_plans.push_back(std::move(keep));
            *status = BBC_OK;
            return g_plans.back().get();
        }
    }
    std::unique_ptr<Plan> p;
    *status = build_plan(n, gs, T, p);
    if (*status != BBC_OK) return nullptr;
    g_plans.push_back(std::move(p));
    while (g_plans.size() > kMaxPlans) g_plans.erase(g_plans.begin());
    return g_plans.back().get();
}

// Replays a plan ordered after `st` and waits for it; fills balanced[] (and the
// elapsed device time in ms when `ms` is given).
bbc_status run_plan(Plan *p, uint64_t *balanced, cudaStream_t st, float *ms) {
    BBC_CUDA_TRY(cudaEventRecord(p->ev_in, st));
    BBC_CUDA_TRY(cudaStreamWaitEvent(p->stream, p->ev_in, 0));
    struct Events {
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        ~Events() {
            if (t0) cudaEventDestroy(t0);
            if (t1) cudaEventDestroy(t1);
        }
    } ev;
    cudaEvent_t &t0 = ev.t0, &t1 = ev.t1;
    if (ms) {
        BBC_CUDA_TRY(cudaEventCreate(&t0));
        BBC_CUDA_TRY(cudaEventCreate(&t1));
        BBC_CUDA_TRY(cudaEventRecord(t0, p->stream));
    }
    if (profiling_active()) {
        // the same work launched directly, so that the kernels' event brackets apply
        BBC_CUDA_TRY(cudaMemsetAsync(p->totals, 0, sizeof(unsigned long long) * 2 * (size_t)p->n,
                                     p->stream));
        BBC_CUDA_TRY(cudaMemsetAsync(p->queue, 0, sizeof(QueueState), p->stream));
        for (const bbc_graph *cg : p->cs_graphs) BBC_TRY(clear_centre_split(cg, p->stream));
        BBC_TRY(launch_count(p->launch, p->stream));
        BBC_CUDA_TRY(cudaMemcpyAsync(p->host_totals, p->totals,
                                     sizeof(unsigned long long) * 2 * (size_t)p->n,
                                     cudaMemcpyDeviceToHost, p->stream));
        BBC_CUDA_TRY(cudaMemcpyAsync(host_error_word(p), &p->queue->error, sizeof(unsigned),
                                     cudaMemcpyDeviceToHost, p->stream));
    } else {
        BBC_CUDA_TRY(cudaGraphLaunch(p->exec, p->stream));
    }
    if (ms) BBC_CUDA_TRY(cudaEventRecord(t1, p->stream));
    BBC_CUDA_TRY(cudaEventRecord(p->ev_out, p->stream));
    BBC_CUDA_TRY(cudaStreamWaitEvent(st, p->ev_out, 0));
    BBC_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (*host_error_word(p)) {
        set_error("counting kernel reported an internal inconsistency");
        return BBC_E_CUDA;
    }
    if (ms) BBC_CUDA_TRY(cudaEventElapsedTime(ms, t0, t1));
    if (balanced)
        for (int i = 0; i < p->n; ++i) balanced[i] = p->host_totals[2 * i];
    return BBC_OK;
}

bbc_status check_graphs(int32_t n, bbc_graph *const *gs) {
    if (n < 0 || (n > 0 && !gs)) {
        set_error("bbc_count_batch: bad graph list");
        return BBC_E_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (!gs[i]) {
            set_error("bbc_count_batch: NULL graph in the list");
            return BBC_E_INVALID_ARG;
        }
    return BBC_OK;
}

Tuning batch_tuning(int32_t n, bbc_graph *const *gs, const bbc_tuning *t) {
    Tuning T = resolve_tuning(t, device_sm_count());
    if (!t) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_tune_cache_locked();
        auto it = g_tuned.find(shape_key(n, gs));
        if (it != g_tuned.end()) T = it->second;
    }
    if (T.split_wedges == 0) {
        uint64_t w = 0;
        for (int i = 0; i < n; ++i) w += gs[i]->wedges;
        T.split_wedges = auto_split(w, device_sm_count(), T.blocks_per_sm);
    }
    if (T.plain) {
        T.warp_max_wedges = 0;
        T.split_wedges = (long long)1 << 62;
    }
    return T;
}

}  // namespace

bbc_status concat_items(const std::vector<CopyJob> &jobs, bool tiles, void *dst, CopyJob *djobs,
                        cudaStream_t st) {
    if (jobs.empty()) return BBC_OK;
    BBC_CUDA_TRY(cudaMemcpyAsync(djobs, jobs.data(), sizeof(CopyJob) * jobs.size(),
                                 cudaMemcpyHostToDevice, st));
    note_launch();
    if (tiles)
        k_concat_items<TileItem><<<(unsigned)jobs.size(), kThreads, 0, st>>>(djobs, static_cast<TileItem *>(dst));
    else
        k_concat_items<HashItem><<<(unsigned)jobs.size(), kThreads, 0, st>>>(djobs, static_cast<HashItem *>(dst));
    BBC_CUDA_TRY(cudaGetLastError());
    return BBC_OK;
}

bbc_status count_batch_impl(int32_t n, bbc_graph *const *gs, uint64_t *balanced,
                            const bbc_tuning *tuning, cudaStream_t st, float *ms) {
    BBC_TRY(check_graphs(n, gs));
    if (n == 0) return BBC_OK;
    const Tuning T = batch_tuning(n, gs, tuning);
    bbc_status s = BBC_OK;
    Plan *p = find_or_build(n, gs, T, &s);
    if (!p) return s;
    return run_plan(p, balanced, st, ms);
}

}  // namespace bbc

using namespace bbc;

extern "C" {

bbc_status bbc_count_batch(int32_t n, bbc_graph *const *gs, uint64_t *balanced,
                           const bbc_tuning *tuning, void *cuda_stream) {
    if (!balanced && n > 0) {
        set_error("bbc_count_batch: NULL output");
        return BBC_E_INVALID_ARG;
    }
    try {
        return count_batch_impl(n, gs, balanced, tuning, static_cast<cudaStream_t>(cuda_stream),
                                nullptr);
    } catch (...) {
        set_error("unexpected exception in bbc_count_batch");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_autotune_batch(int32_t n, bbc_graph *const *gs, bbc_tuning *best,
                              void *cuda_stream) {
    if (!best) return BBC_E_INVALID_ARG;
    try {
        BBC_TRY(check_graphs(n, gs));
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        // coordinate search from the defaults: each knob in turn over its candidates,
        // keeping the fastest value before moving to the next knob
        std::vector<uint64_t> ref(std::max(n, 1)), got(std::max(n, 1));
        bool have_ref = false;
        auto timed = [&](const bbc_tuning &t, float *out_ms) -> bbc_status {
            float ms_best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                float ms = 0.f;
                BBC_TRY(count_batch_impl(n, gs, got.data(), &t, st, &ms));
                if (rep > 0) ms_best = std::min(ms_best, ms);
            }
            if (!have_ref) {
                ref = got;
                have_ref = true;
            } else if (ref != got) {
                set_error("bbc_autotune_batch: candidates disagree on the counts");
                return BBC_E_CUDA;
            }
            *out_ms = ms_best;
            return BBC_OK;
        };
        uint64_t wsum = 0;
        for (int i = 0; i < n; ++i) wsum += gs[i]->wedges;
        const long long s_auto = auto_split(wsum, device_sm_count(), 2);
        bbc_tuning best_t{};
        best_t.blocks_per_sm = 2;
        best_t.warp_max_wedges = 256;
        best_t.queue_chunk = 1;
        best_t.group_warps = 4;
        float best_ms = 1e30f;
        BBC_TRY(timed(best_t, &best_ms));
        const std::vector<int> knob_tiles = {0, 16384, 8192, 4096};
        const std::vector<int> knob_warp = {64, 256, 512};
        const std::vector<int> knob_blocks = {1, 2};
        const std::vector<int> knob_chunk = {1, 4, 16};
        const std::vector<int> knob_group = {4, 8};
        const std::vector<long long> knob_split = {s_auto / 4, s_auto, 4 * s_auto};
        auto sweep = [&](auto values, auto set) -> bbc_status {
            bbc_tuning keep = best_t;
            for (auto v : values) {
                bbc_tuning t = keep;
                set(t, v);
                if (memcmp(&t, &keep, sizeof t) == 0) continue;
                float ms = 0.f;
                BBC_TRY(timed(t, &ms));
                if (ms < best_ms) {
                    best_ms = ms;
                    best_t = t;
                }
            }
            return BBC_OK;
        };
        BBC_TRY(sweep(knob_group, [](bbc_tuning &t, int v) { t.group_warps = v; }));
        BBC_TRY(sweep(knob_tiles, [](bbc_tuning &t, int v) { t.tile_words = v; }));
        BBC_TRY(sweep(knob_warp, [](bbc_tuning &t, int v) { t.warp_max_wedges = v; }));
        BBC_TRY(sweep(knob_split, [](bbc_tuning &t, long long v) {
            t.split_wedges = (int32_t)std::min<long long>(std::max<long long>(v, 1), INT32_MAX);
        }));
        BBC_TRY(sweep(knob_blocks, [](bbc_tuning &t, int v) { t.blocks_per_sm = v; }));
        BBC_TRY(sweep(knob_chunk, [](bbc_tuning &t, int v) { t.queue_chunk = v; }));
        *best = best_t;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            load_tune_cache_locked();
            g_tuned[shape_key(n, gs)] = resolve_tuning(&best_t, device_sm_count());
            save_tune_cache_locked();
        }
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_autotune_batch");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_batch_tuning(int32_t n, bbc_graph *const *gs, bbc_tuning *out) {
    if (!out) return BBC_E_INVALID_ARG;
    try {
        BBC_TRY(check_graphs(n, gs));
        const Tuning T = batch_tuning(n, gs, nullptr);
        memset(out, 0, sizeof *out);
        out->tile_words = T.tile_words;
        out->warp_max_wedges = T.warp_max_wedges;
        out->dense_min_permille = T.dense_min_permille;
        out->split_wedges = (int32_t)std::min<long long>(T.split_wedges, INT32_MAX);
        out->blocks_per_sm = T.blocks_per_sm;
        out->plain = T.plain;
        out->queue_chunk = T.queue_chunk;
        out->group_warps = T.group_warps;
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_batch_tuning");
        return BBC_E_CUDA;
    }
}

}  // extern "C"
