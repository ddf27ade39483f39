// api.cu -- the extern "C" entry points of include/bbc.h for single graphs, plus the
// library's error state, memory pool and tuning defaults.
#include <algorithm>
#include <atomic>
#include <vector>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "graph.cuh"

namespace bbc {
namespace {

thread_local std::string g_last_error = "no error";

struct PoolEntry {
    cudaMemPool_t pool = nullptr;
    int sms = 0;
};
std::mutex g_pool_mu;
PoolEntry g_pools[64];

PoolEntry *device_entry() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    PoolEntry &e = g_pools[dev];
    if (!e.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&e.pool, &props) != cudaSuccess) {
            e.pool = nullptr;
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;  // keep freed blocks for reuse within this process
        cudaMemPoolSetAttribute(e.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaDeviceGetAttribute(&e.sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return &e;
}

// The descriptor travels as a kernel argument, so queuing it never waits on the stream.
__global__ void k_store_descriptor(DevGraph d, DevGraph *dst) { *dst = d; }

__global__ void k_scatter_per_vertex(const unsigned long long *__restrict__ by_rank,
                                     const int32_t *__restrict__ perm, int64_t n,
                                     unsigned long long *__restrict__ out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        out[perm[r]] = by_rank[r];
}

}  // namespace

// Wedges and pair-side edges of the anchors behind a work list (one entry per anchor:
// a tile anchor's first item (tile 0, part 0 when centre-split), or its single hash /
// warp-tile / group-tile item).
__global__ void k_work_tile(const TileItem *__restrict__ items, int n, const int64_t *__restrict__ rowS_off,
                            const unsigned long long *__restrict__ wl, const CentreSplit *__restrict__ cs_desc,
                            unsigned long long *__restrict__ out) {
    unsigned long long w = 0, e = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const TileItem it = items[i];
        if (is_centre_split(it)) {
            const CentreSplit d = cs_desc[it.tile_begin];
            if (d.tile != 0 || d.part != 0) continue;
        } else if (it.tile_begin != 0) {
            continue;
        }
        w += wl[it.anchor];
        e += (unsigned long long)(rowS_off[it.anchor + 1] - rowS_off[it.anchor]);
    }
    if (w) atomicAdd(out, w);
    if (e) atomicAdd(out + 1, e);
}

__global__ void k_work_hash(const HashItem *__restrict__ items, int n, const int64_t *__restrict__ rowS_off,
                            const unsigned long long *__restrict__ wl, unsigned long long *__restrict__ out) {
    unsigned long long w = 0, e = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const HashItem it = items[i];
        w += wl[it.anchor];
        e += (unsigned long long)(rowS_off[it.anchor + 1] - rowS_off[it.anchor]);
    }
    if (w) atomicAdd(out, w);
    if (e) atomicAdd(out + 1, e);
}

// Fails unless the current device is a usable GB300 (compute capability 10.3).
bbc_status check_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("no CUDA device: ") + cudaGetErrorString(e));
        return BBC_E_NO_DEVICE;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) {
        char buf[128];
        snprintf(buf, sizeof buf, "device %d is sm_%d%d; this library is built for sm_103a", dev,
                 major, minor);
        set_error(buf);
        return BBC_E_NO_DEVICE;
    }
    return BBC_OK;
}

void set_error(const std::string &msg) { g_last_error = msg; }

namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
struct ProfSlot {
    cudaEvent_t a = nullptr, b = nullptr;
    int kind = 0;
    bool used = false;
};
std::vector<ProfSlot> g_prof;
const char *const kProfNames[kProfKinds] = {"k_tile", "k_warp_hash", "k_warp_tile", "k_group_tile",
                                            "k_tile_motif", "k_tile_cs"};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool profiling_active() { return g_prof_on.load(std::memory_order_relaxed); }

int profile_begin(int kind, cudaStream_t st) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfSlot sl;
    if (cudaEventCreate(&sl.a) != cudaSuccess || cudaEventCreate(&sl.b) != cudaSuccess) return -1;
    sl.kind = kind;
    cudaEventRecord(sl.a, st);
    g_prof.push_back(sl);
    return (int)g_prof.size() - 1;
}

void profile_end(int token, cudaStream_t st) {
    if (token < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (token >= (int)g_prof.size()) return;
    cudaEventRecord(g_prof[token].b, st);
    g_prof[token].used = true;
}

bbc_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return BBC_E_NO_MEMORY;
    return BBC_E_CUDA;
}

bbc_status dev_alloc(void **p, size_t bytes, cudaStream_t st) {
    PoolEntry *e = device_entry();
    if (!e) {
        set_error("could not create the device memory pool");
        return BBC_E_CUDA;
    }
    cudaError_t err = cudaMallocFromPoolAsync(p, bytes, e->pool, st);
    if (err != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cuda_fail(err, "cudaMallocFromPoolAsync");
    }
    return BBC_OK;
}

void dev_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

size_t l2_bytes() {
    static thread_local int dev_cached = -1;
    static thread_local size_t bytes = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (size_t)128 << 20;
    if (dev != dev_cached) {
        int v = 0;
        bytes = cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) == cudaSuccess && v > 0
                    ? (size_t)v
                    : (size_t)128 << 20;
        dev_cached = dev;
    }
    return bytes;
}

bool rows_exceed_l2(const bbc_graph *g) { return (size_t)g->n_edges * 4 > l2_bytes(); }

int device_sm_count() {
    PoolEntry *e = device_entry();
    if (e && e->sms > 0) return e->sms;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
        return sms;
    return 152;  // GB300
}

Tuning resolve_tuning(const bbc_tuning *t, int sm_count) {
    (void)sm_count;
    Tuning r;
    r.tile_words = 0;  // 0: the largest tile that keeps blocks_per_sm blocks resident
    r.warp_max_wedges = 256;
    r.dense_min_permille = 0;
    r.split_wedges = 0;  // 0: chosen per launch from the total work
    r.blocks_per_sm = 2;
    r.plain = 0;
    r.queue_chunk = 1;
    r.group_warps = kGroupWarps;
    if (t) {
        if (t->group_warps == 8) r.group_warps = 8;
        if (t->queue_chunk > 0) r.queue_chunk = t->queue_chunk < 64 ? t->queue_chunk : 64;
        r.plain = t->plain ? 1 : 0;
        if (t->blocks_per_sm == 1 || t->blocks_per_sm == 2) r.blocks_per_sm = t->blocks_per_sm;
        if (t->tile_words > 0) r.tile_words = t->tile_words;
        if (t->warp_max_wedges > 0) r.warp_max_wedges = t->warp_max_wedges;
        if (t->dense_min_permille > 0) r.dense_min_permille = t->dense_min_permille;
        if (t->split_wedges > 0) r.split_wedges = t->split_wedges;
    }
    // limits: tiles are whole 32-byte groups and fit the shared memory an SM gives each
    // of blocks_per_sm resident blocks (228 KB per SM, 1 KB reserved per block, minus
    // the kernel's static shared memory); hash tables hold at most 512 wedges
    const int per_block = (228 * 1024) / r.blocks_per_sm - 1024 - tile_static_smem_bytes();
    const int cap = std::min(per_block, 227 * 1024 - tile_static_smem_bytes()) / 4 - kTileSlackWords;
    if (r.tile_words == 0 || r.tile_words > cap) r.tile_words = cap;
    if (r.tile_words < 1024) r.tile_words = 1024;
    r.tile_words &= ~7;
    if (r.warp_max_wedges > 512) r.warp_max_wedges = 512;
    return r;
}

// Splits anchors whose wedge count exceeds a fair share of one block's work.
long long auto_split(uint64_t wedges, int sm_count, int blocks_per_sm) {
    const long long blocks = (long long)sm_count * blocks_per_sm;
    long long s = (long long)(wedges / (uint64_t)(blocks * 4 > 0 ? blocks * 4 : 1));
    if (s < (1ll << 22)) s = 1ll << 22;
    return s;
}

bbc_status count_graph(bbc_graph *g, uint64_t *totals_dev, uint64_t *per_u, uint64_t *per_v,
                       const bbc_tuning *tuning, cudaStream_t st) {
    Tuning T = resolve_tuning(tuning, device_sm_count());
    if (T.split_wedges == 0) T.split_wedges = auto_split(g->wedges, device_sm_count(), T.blocks_per_sm);
    if (T.plain) {
        T.warp_max_wedges = 0;
        T.split_wedges = (long long)1 << 62;
    }
    BBC_TRY(build_work_lists(g, T, st));
    const bool pv = per_u || per_v;
    if (pv && !g->bS) {
        BBC_TRY(dev_alloc_n(&g->bS, (size_t)g->nS, st));
        BBC_TRY(dev_alloc_n(&g->bC, (size_t)g->nC, st));
        g->device_bytes += (size_t)(g->nS + g->nC) * 8;
    }
    if (pv) {
        if (g->nS) BBC_CUDA_TRY(cudaMemsetAsync(g->bS, 0, (size_t)g->nS * 8, st));
        if (g->nC) BBC_CUDA_TRY(cudaMemsetAsync(g->bC, 0, (size_t)g->nC * 8, st));
    }
    BBC_CUDA_TRY(cudaMemsetAsync(g->totals, 0, 16, st));
    BBC_CUDA_TRY(cudaMemsetAsync(g->queue, 0, sizeof(QueueState), st));
    BBC_TRY(clear_centre_split(g, st));
    static_assert(sizeof(DevGraph) % 8 == 0, "descriptor layout");
    DevGraph d = host_descriptor(g, pv, true);
    note_launch();
    k_store_descriptor<<<1, 1, 0, st>>>(d, g->dgraph);
    BBC_CUDA_TRY(cudaGetLastError());
    CountLaunch L{};
    L.graphs = g->dgraph;
    L.tile_items = g->tile_items;
    L.n_tile_items = g->n_tile;
    L.warp_items = g->warp_items;
    L.n_warp_items = g->n_warp;
    L.wt_items = g->wt_items;
    L.n_wt_items = g->n_wt;
    L.gt_items = g->gt_items;
    L.n_gt_items = g->n_gt;
    L.queue = g->queue;
    L.tuning = T;
    L.prefetch = rows_exceed_l2(g);
    if (pv) {
        L.cs_items = g->cs_items;
        L.n_cs_items = g->n_cs_items;
        L.per_vertex = true;
    }
    BBC_TRY(launch_count(L, st));
    if (pv) {
        uint64_t *outS = g->side == 0 ? per_u : per_v;
        uint64_t *outC = g->side == 0 ? per_v : per_u;
        if (outS && g->nS) {
            note_launch();
            k_scatter_per_vertex<<<(unsigned)std::min<int64_t>((g->nS + 255) / 256, 4096), 256, 0, st>>>(
                g->bS, g->permS, g->nS, reinterpret_cast<unsigned long long *>(outS));
            BBC_CUDA_TRY(cudaGetLastError());
        }
        if (outC && g->nC) {
            note_launch();
            k_scatter_per_vertex<<<(unsigned)std::min<int64_t>((g->nC + 255) / 256, 4096), 256, 0, st>>>(
                g->bC, g->permC, g->nC, reinterpret_cast<unsigned long long *>(outC));
            BBC_CUDA_TRY(cudaGetLastError());
        }
    }
    if (totals_dev && totals_dev != reinterpret_cast<uint64_t *>(g->totals))
        BBC_CUDA_TRY(cudaMemcpyAsync(totals_dev, g->totals, 16, cudaMemcpyDeviceToDevice, st));
    return BBC_OK;
}

}  // namespace bbc

using namespace bbc;

extern "C" {

const char *bbc_status_string(bbc_status st) {
    switch (st) {
        case BBC_OK: return "ok";
        case BBC_E_INVALID_ARG: return "invalid argument";
        case BBC_E_OUT_OF_RANGE: return "vertex id out of range";
        case BBC_E_BAD_SIGN: return "sign is not +1 or -1";
        case BBC_E_DUPLICATE_EDGE: return "duplicate edge";
        case BBC_E_OVERFLOW_RISK: return "count could overflow 64 bits";
        case BBC_E_NO_MEMORY: return "out of memory";
        case BBC_E_OVER_BUDGET: return "request exceeds the device memory budget";
        case BBC_E_CUDA: return "CUDA error";
        case BBC_E_TIMEOUT: return "timed out";
        case BBC_E_CANCELLED: return "cancelled";
        case BBC_E_NOT_READY: return "not ready";
        case BBC_E_NO_DEVICE: return "no usable sm_103 device";
    }
    return "unknown status";
}

const char *bbc_last_error(void) { return bbc::g_last_error.c_str(); }

bbc_status bbc_tuning_default(bbc_tuning *t) {
    if (!t) return BBC_E_INVALID_ARG;
    const Tuning r = resolve_tuning(nullptr, 0);
    memset(t, 0, sizeof *t);
    t->tile_words = r.tile_words;
    t->warp_max_wedges = r.warp_max_wedges;
    t->dense_min_permille = r.dense_min_permille;
    t->split_wedges = 0;
    t->blocks_per_sm = r.blocks_per_sm;
    t->plain = 0;
    t->queue_chunk = r.queue_chunk;
    t->group_warps = r.group_warps;
    return BBC_OK;
}

bbc_status bbc_prepare(int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *u,
                       const int32_t *v, const int8_t *sign, uint32_t flags, void *cuda_stream,
                       bbc_graph **out) {
    try {
        if (!out || n_u < 0 || n_v < 0 || n_edges < 0) {
            set_error("bbc_prepare: NULL output or negative size");
            return BBC_E_INVALID_ARG;
        }
        if (n_edges > 0 && (!u || !v || !sign)) {
            set_error("bbc_prepare: NULL edge array");
            return BBC_E_INVALID_ARG;
        }
        if ((flags & BBC_SIDE_FORCE_U) && (flags & BBC_SIDE_FORCE_V)) {
            set_error("bbc_prepare: both side flags set");
            return BBC_E_INVALID_ARG;
        }
        if (n_edges >= (int64_t)INT32_MAX || (int64_t)n_u + 1 >= (int64_t)INT32_MAX ||
            (int64_t)n_v + 1 >= (int64_t)INT32_MAX) {
            set_error("bbc_prepare: sizes must stay below 2^31 - 1");
            return BBC_E_INVALID_ARG;
        }
        BBC_TRY(check_device());
        return prepare_graph(n_u, n_v, n_edges, u, v, sign, flags,
                             static_cast<cudaStream_t>(cuda_stream), out);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return BBC_E_NO_MEMORY;
    } catch (...) {
        set_error("unexpected exception in bbc_prepare");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_count_async(bbc_graph *g, uint64_t *totals_dev, uint64_t *per_u, uint64_t *per_v,
                           const bbc_tuning *tuning, void *cuda_stream) {
    if (!g) {
        set_error("bbc_count_async: NULL graph");
        return BBC_E_INVALID_ARG;
    }
    try {
        return count_graph(g, totals_dev, per_u, per_v, tuning,
                           static_cast<cudaStream_t>(cuda_stream));
    } catch (...) {
        set_error("unexpected exception in bbc_count_async");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_count(bbc_graph *g, uint64_t *balanced, uint64_t *unbalanced, uint64_t *per_u,
                     uint64_t *per_v, const bbc_tuning *tuning, void *cuda_stream) {
    if (!g || !balanced) {
        set_error("bbc_count: NULL graph or NULL balanced");
        return BBC_E_INVALID_ARG;
    }
    try {
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        BBC_TRY(count_graph(g, nullptr, per_u, per_v, tuning, st));
        unsigned long long host[2] = {0, 0};
        QueueState q{};
        BBC_CUDA_TRY(cudaMemcpyAsync(host, g->totals, 16, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaMemcpyAsync(&q, g->queue, sizeof q, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        if (q.error) {
            set_error("counting kernel reported an internal inconsistency");
            return BBC_E_CUDA;
        }
        *balanced = host[0];
        if (unbalanced) *unbalanced = host[1];
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_count");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_count_motif(bbc_graph *g, int32_t kind, int32_t k, uint64_t *out, void *cuda_stream) {
    if (!g || !out) {
        set_error("bbc_count_motif: NULL graph or NULL output");
        return BBC_E_INVALID_ARG;
    }
    if (kind != BBC_MOTIF_SIGN_CLASSES && kind != BBC_MOTIF_BICLIQUE_2K) {
        set_error("bbc_count_motif: unknown motif kind");
        return BBC_E_INVALID_ARG;
    }
    if (kind == BBC_MOTIF_BICLIQUE_2K && (k < 2 || k == INT32_MAX)) {
        set_error("bbc_count_motif: k must lie in [2, 2^31 - 2]");
        return BBC_E_INVALID_ARG;
    }
    try {
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        const int sms = device_sm_count();
        Tuning T = resolve_tuning(nullptr, sms);
        T.split_wedges = auto_split(g->wedges, sms, T.blocks_per_sm);
        T.warp_max_wedges = 0;  // no hash path: every anchor with wedges is a tile item
        T.tiles_only = 1;
        const int smem_words = T.tile_words;
        // class counters take twice the words per endpoint: the lists see half the tile
        if (kind == BBC_MOTIF_SIGN_CLASSES) T.tile_words = smem_words / 2;
        BBC_TRY(build_work_lists(g, T, st));
        unsigned long long *dout = nullptr;
        BBC_TRY(dev_alloc_n(&dout, 8, st));
        bbc_status rc = BBC_OK;
        unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        do {
            cudaError_t e = cudaMemsetAsync(dout, 0, 64, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(g->queue, 0, sizeof(QueueState), st);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "bbc_count_motif");
                break;
            }
            DevGraph d = host_descriptor(g, false, true);
            note_launch();
            k_store_descriptor<<<1, 1, 0, st>>>(d, g->dgraph);
            if ((e = cudaGetLastError()) != cudaSuccess) {
                rc = cuda_fail(e, "bbc_count_motif");
                break;
            }
            const int blocks = std::max(1, std::min(g->n_tile, sms * T.blocks_per_sm));
            rc = launch_motif(g->dgraph, g->tile_items, g->n_tile, &g->queue->tile_head, kind, k,
                              smem_words, blocks, dout, st);
            if (rc != BBC_OK) break;
            e = cudaMemcpyAsync(h, dout, 64, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_fail(e, "bbc_count_motif");
        } while (false);
        dev_free(dout, st);
        if (rc != BBC_OK) return rc;
        if (h[7]) {
            set_error("bbc_count_motif: a count exceeds 2^64 - 1");
            return BBC_E_OVERFLOW_RISK;
        }
        const int n_out = kind == BBC_MOTIF_SIGN_CLASSES ? 6 : 2;
        for (int j = 0; j < n_out; ++j) out[j] = h[j];
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_count_motif");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_graph_work(bbc_graph *g, uint64_t *out, void *cuda_stream) {
    if (!g || !out) {
        set_error("bbc_graph_work: NULL graph or NULL output");
        return BBC_E_INVALID_ARG;
    }
    try {
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        if (!g->items_valid) {
            const int sms = device_sm_count();
            Tuning T = resolve_tuning(nullptr, sms);
            T.split_wedges = auto_split(g->wedges, sms, T.blocks_per_sm);
            BBC_TRY(build_work_lists(g, T, st));
        }
        unsigned long long *d = nullptr;
        BBC_TRY(dev_alloc_n(&d, 8, st));
        bbc_status rc = BBC_OK;
        unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        cudaError_t e = cudaMemsetAsync(d, 0, 64, st);
        const int nl[4] = {g->n_tile, g->n_gt, g->n_wt, g->n_warp};
        if (e == cudaSuccess && g->n_tile > 0) {
            note_launch();
            k_work_tile<<<std::min((g->n_tile + 255) / 256, 1024), 256, 0, st>>>(g->tile_items, g->n_tile,
                                                                                  g->rowS_off, g->wl, g->cs_desc, d);
        }
        const HashItem *lists[3] = {g->gt_items, g->wt_items, g->warp_items};
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            if (nl[k + 1] > 0) {
                note_launch();
                k_work_hash<<<std::min((nl[k + 1] + 255) / 256, 1024), 256, 0, st>>>(lists[k], nl[k + 1],
                                                                                    g->rowS_off, g->wl, d + 2 * (k + 1));
            }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 64, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "bbc_graph_work");
        dev_free(d, st);
        if (rc != BBC_OK) return rc;
        for (int k = 0; k < 4; ++k) {
            out[3 * k] = (uint64_t)nl[k];
            out[3 * k + 1] = h[2 * k];
            out[3 * k + 2] = h[2 * k + 1];
        }
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_graph_work");
        return BBC_E_CUDA;
    }
}

unsigned long long bbc_launch_count(void) { return g_launches.load(); }

bbc_status bbc_profile_start(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (ProfSlot &sl : g_prof) {
        cudaEventDestroy(sl.a);
        cudaEventDestroy(sl.b);
    }
    g_prof.clear();
    g_prof_on.store(true);
    return BBC_OK;
}

bbc_status bbc_profile_stop(bbc_kernel_time *out, int32_t capacity, int32_t *count) {
    g_prof_on.store(false);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    long long launches[kProfKinds] = {0};
    double ms[kProfKinds] = {0};
    bbc_status st = BBC_OK;
    for (ProfSlot &sl : g_prof) {
        if (sl.used) {
            cudaError_t e = cudaEventSynchronize(sl.b);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, sl.a, sl.b);
            if (e != cudaSuccess) st = cuda_fail(e, "bbc_profile_stop");
            launches[sl.kind] += 1;
            ms[sl.kind] += t;
        }
        cudaEventDestroy(sl.a);
        cudaEventDestroy(sl.b);
    }
    g_prof.clear();
    int n = 0;
    for (int k = 0; k < kProfKinds; ++k) {
        if (!launches[k]) continue;
        if (out && n < capacity) {
            out[n].name = kProfNames[k];
            out[n].launches = launches[k];
            out[n].total_ms = ms[k];
        }
        ++n;
    }
    if (count) *count = n;
    return st;
}

bbc_status bbc_memory_usage(size_t *used, size_t *used_high, int32_t reset_high) {
    PoolEntry *e = device_entry();
    if (!e) {
        set_error("bbc_memory_usage: no device memory pool");
        return BBC_E_CUDA;
    }
    uint64_t cur = 0, high = 0;
    BBC_CUDA_TRY(cudaMemPoolGetAttribute(e->pool, cudaMemPoolAttrUsedMemCurrent, &cur));
    BBC_CUDA_TRY(cudaMemPoolGetAttribute(e->pool, cudaMemPoolAttrUsedMemHigh, &high));
    if (used) *used = (size_t)cur;
    if (used_high) *used_high = (size_t)high;
    if (reset_high) {
        uint64_t zero = 0;
        BBC_CUDA_TRY(cudaMemPoolSetAttribute(e->pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    return BBC_OK;
}

bbc_status bbc_graph_info(const bbc_graph *g, int32_t *side, uint64_t *wedges,
                          size_t *device_bytes, int64_t *n_edges) {
    if (!g) return BBC_E_INVALID_ARG;
    if (side) *side = g->side;
    if (wedges) *wedges = g->wedges;
    if (device_bytes) *device_bytes = g->device_bytes;
    if (n_edges) *n_edges = g->n_edges;
    return BBC_OK;
}

void bbc_graph_free(bbc_graph *g) {
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    const int dev = g->device;  // release_graph deletes g
    if (prev != dev) cudaSetDevice(dev);
    release_graph(g, nullptr);
    cudaStreamSynchronize(nullptr);
    if (prev != dev) cudaSetDevice(prev);
}

}  // extern "C"
