// noalloc.cu -- bbc_count_noalloc: the counting step of a prepared graph with every
// piece of per-call scratch in one static device array, for callers that cannot
// allocate device memory at the time they count.
//
// The array below is a file-scope __device__ object: each GPU that loads the library
// holds it (1 MiB) until the process exits. Host code cannot use its name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.
#include <cstdio>
#include <mutex>

#include "graph.cuh"

namespace bbc {
namespace {

constexpr size_t kNoallocBytes = size_t(1) << 20;
constexpr size_t kHeaderBytes = 256;

struct NoallocHeader {
    QueueState queue;
    DevGraph graph;
};
static_assert(sizeof(NoallocHeader) <= kHeaderBytes, "header must fit its 256-byte slot");

// One work item per anchor follows the header.
constexpr int kNoallocMaxAnchors = (int)((kNoallocBytes - kHeaderBytes) / sizeof(TileItem));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_addr_mu;
void *g_addr[64] = {};

// Clears the queue and the caller's totals, and stores the descriptor (no per-vertex
// output on this path) with its totals pointing at the caller's buffer.
__global__ void k_noalloc_setup(DevGraph d, NoallocHeader *h, unsigned long long *totals) {
    d.bS = nullptr;
    d.bC = nullptr;
    d.totals = totals;
    h->graph = d;
    h->queue.tile_head = 0;
    h->queue.warp_head = 0;
    h->queue.cs_head = 0;
    h->queue.error = 0;
    totals[0] = 0;
    totals[1] = 0;
}

// Item a covers every endpoint tile of anchor a (rank order, heaviest first). Anchors
// that close no butterfly get an empty tile range.
__global__ void k_noalloc_items(const unsigned long long *__restrict__ wl,
                                const int64_t *__restrict__ rowS_off, int nS, int orient_low,
                                int tile_words, TileItem *__restrict__ items) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nS; a += (int64_t)gridDim.x * blockDim.x) {
        const long long w = (long long)wl[a];
        const long long deg = rowS_off[a + 1] - rowS_off[a];
        int nt = 0, cw = 0;
        if (w > 0 && deg >= 2) {
            const long long maxcount = deg < w ? deg : w;
            cw = maxcount <= 255 ? 0 : (maxcount <= 65535 ? 1 : 2);
            const long long ept = cw == 0 ? 2ll * tile_words : (cw == 1 ? tile_words : tile_words / 2);
            const long long span = orient_low ? a : (long long)nS - 1 - a;
            nt = (int)((span + ept - 1) / ept);
        }
        items[a] = TileItem{0, (int32_t)a, 0, pack_tile_end(nt, cw)};
    }
}

bbc_status scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (dev < 0 || dev >= 64) {
        set_error("bbc_count_noalloc: device index out of range");
        return BBC_E_INVALID_ARG;
    }
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return BBC_OK;
}

}  // namespace
}  // namespace bbc

using namespace bbc;

extern "C" bbc_status bbc_count_noalloc(const bbc_graph *g, uint64_t *totals_dev, void *cuda_stream) {
    if (!g || !totals_dev) {
        set_error("bbc_count_noalloc: NULL graph or NULL totals");
        return BBC_E_INVALID_ARG;
    }
    if (g->nS > kNoallocMaxAnchors) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "bbc_count_noalloc: the graph has %d pair-side vertices; the static scratch "
                 "holds work for at most %d",
                 g->nS, kNoallocMaxAnchors);
        set_error(buf);
        return BBC_E_INVALID_ARG;
    }
    int dev = 0;
    BBC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != g->device) {
        set_error("bbc_count_noalloc: the graph was prepared on another device");
        return BBC_E_INVALID_ARG;
    }
    unsigned char *base = nullptr;
    BBC_TRY(scratch_address(dev, &base));
    NoallocHeader *hdr = reinterpret_cast<NoallocHeader *>(base);
    TileItem *items = reinterpret_cast<TileItem *>(base + kHeaderBytes);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const Tuning T = resolve_tuning(nullptr, 0);
    int sms = 0;
    BBC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevGraph d = host_descriptor(g, false);
    note_launch();
    k_noalloc_setup<<<1, 1, 0, st>>>(d, hdr, reinterpret_cast<unsigned long long *>(totals_dev));
    BBC_CUDA_TRY(cudaGetLastError());
    if (g->nS > 0) {
        const int blocks = (g->nS + 255) / 256;
        note_launch();
        k_noalloc_items<<<blocks, 256, 0, st>>>(g->wl, g->rowS_off, g->nS, g->orient_low,
                                                T.tile_words, items);
        BBC_CUDA_TRY(cudaGetLastError());
    }
    return launch_tile_only(&hdr->graph, items, g->nS, &hdr->queue.tile_head, T.tile_words,
                            sms * T.blocks_per_sm, st);
}
