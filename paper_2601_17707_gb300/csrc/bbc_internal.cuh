// bbc_internal.cuh -- device layout, work items and launchers shared by the library's
// translation units. Not part of the public boundary (include/bbc.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bbc.h"

namespace bbc {

constexpr uint32_t kSignBit = 0x80000000u;
constexpr uint32_t kIdMask = 0x7fffffffu;

struct CentreSplit;

// One prepared graph as the counting kernels see it. S is the pair (anchor/endpoint)
// side, C the centre side; both are relabelled by rank (degree descending, id
// descending, Def. 6). Entries pack the neighbour's rank with the edge sign in bit 31
// (set = negative edge).
struct DevGraph {
    const int64_t *rowS_off;   // nS + 1
    const uint32_t *rowS;      // S -> C entries (centre rank | sign)
    const int64_t *rowC_off;   // nC + 1
    const uint32_t *rowC;      // C -> S entries (anchor rank | sign), ascending rank per row
    int32_t nS, nC;
    int32_t orient_low;        // 0: anchor a pairs with endpoints of higher rank (lower
                               // priority); 1: with endpoints of lower rank
    int32_t pad;
    unsigned long long *bS;    // per-vertex balanced counts by S rank (nullable)
    unsigned long long *bC;    // per-vertex balanced counts by C rank (nullable)
    unsigned long long *totals;// [0] balanced, [1] unbalanced
    const unsigned long long *wl; // oriented wedges per anchor rank (orders work items)
    const uint2 *rng;          // per S -> C entry (a, c): the entries of row c that are
                               // endpoints of a, as an index range [x, y) into rowC
    const uint32_t *bnd;       // interior tile boundaries (nullable: found by search);
                               // boundary t (1 <= t < tiles) of entry i of anchor a is
                               // bnd[boff[a] + (t - 1) * degree(a) + i], an index into rowC
    const int64_t *boff;
    // centre-split tiles (items with parts): per tile group, the merged counters
    // (cs_group_words words: p, n of endpoint lo + i at 2 i, 2 i + 1) and an arrival
    // counter; both zeroed before every count launch
    const CentreSplit *cs_desc;
    uint32_t *cs_buf;
    unsigned *cs_arrive;
    int64_t cs_group_words;
};

// A unit of work of the tile kernel: anchor `anchor` of graph `graph`, endpoint tiles
// [tile_begin, tile_end) over the anchor's endpoint range. The top two bits of
// `tile_end_cw` hold the counter width code (0: 8-bit, 1: 16-bit, 2: 32-bit counters),
// which fixes the endpoints per tile (2, 1 or 1/2 per shared-memory word). Bit 29 marks
// a centre-split item: it covers one tile and one part of the anchor's centres, and
// `tile_begin` indexes its CentreSplit record (DevGraph::cs_desc) instead.
struct TileItem {
    int32_t graph;
    int32_t anchor;
    int32_t tile_begin;
    uint32_t tile_end_cw;
};

constexpr uint32_t kCentreSplitBit = 1u << 29;
__host__ __device__ inline int tile_end_of(const TileItem &t) { return (int)(t.tile_end_cw & 0x1fffffffu); }
__host__ __device__ inline int tile_width_of(const TileItem &t) { return (int)(t.tile_end_cw >> 30); }
__host__ __device__ inline bool is_centre_split(const TileItem &t) { return (t.tile_end_cw & kCentreSplitBit) != 0; }

// One part of a centre-split tile: tile `tile` of the anchor, centres [part / parts,
// (part + 1) / parts) of its S -> C row (by position), merged through tile group `group`.
struct CentreSplit {
    int32_t tile;
    int16_t part, parts;
    int32_t group;
    int32_t pad;
};
// Most parts of one centre-split tile.
constexpr int kMaxParts = 64;

// Counter widths of a block tile: 0 two 8-bit, 1 two 16-bit, 2 two 32-bit counters per
// endpoint. A tile item whose width field is kWidthPerTile chooses the width tile by
// tile: a pair (a, w) shares at most min(deg a, wedges of a, deg w) centres, and degrees
// fall with rank, so a tile's first endpoint bounds all its counts.
constexpr int kWidthPerTile = 3;
__host__ __device__ inline int width_for_bound(unsigned long long bound) {
    return bound <= 255 ? 0 : (bound <= 65535 ? 1 : 2);
}
__host__ __device__ constexpr uint32_t tile_endpoints(int cw, uint32_t tile_words) {
    return cw == 0 ? tile_words * 2 : (cw == 1 ? tile_words : tile_words / 2);
}
// Words the tile kernel allocates past tile_words: a tile of 8-bit counters whose first
// endpoint is odd starts one endpoint early (its words hold an even and an odd endpoint),
// and the epilogue reads whole 16-byte groups.
constexpr int kTileSlackWords = 4;

struct VarTile {
    uint32_t lo, hi;   // endpoint ranks [lo, hi)
    int cw;
};
// The tile that starts at endpoint rank lo (< range_hi) of an anchor whose counts are at
// most bound_a.
__device__ __forceinline__ VarTile var_tile_at(const int64_t *__restrict__ rowS_off, unsigned long long bound_a,
                                               uint32_t lo, uint32_t range_hi, uint32_t tile_words) {
    const unsigned long long d = (unsigned long long)(rowS_off[lo + 1] - rowS_off[lo]);
    VarTile t;
    t.lo = lo;
    t.cw = width_for_bound(d < bound_a ? d : bound_a);
    const uint32_t e = tile_endpoints(t.cw, tile_words);
    t.hi = range_hi - lo > e ? lo + e : range_hi;
    return t;
}
__device__ __forceinline__ int var_tile_count(const int64_t *__restrict__ rowS_off, unsigned long long bound_a,
                                              uint32_t range_lo, uint32_t range_hi, uint32_t tile_words) {
    int n = 0;
    for (uint32_t lo = range_lo; lo < range_hi; ++n) lo = var_tile_at(rowS_off, bound_a, lo, range_hi, tile_words).hi;
    return n;
}
__host__ __device__ inline uint32_t pack_tile_end(int end, int cw) {
    return (uint32_t)end | ((uint32_t)cw << 30);
}

// A unit of work of the warp kernels: one anchor, its oriented wedge count, and (warp
// tiles) its counter width code.
struct HashItem {
    int32_t graph;
    int32_t anchor;
    int32_t wedges;
    int32_t cw;
};

// Words of one warp's counter table in the group-tile kernel (a group of gw warps pools
// gw tables), and the endpoints such a table holds per counter width code.
constexpr int kWtWords = 1536;
constexpr int kGroupWarps = 4;
__host__ __device__ constexpr uint32_t group_tile_endpoints(int gw, int cw) {
    return cw == 0 ? 2u * kWtWords * gw
                   : (cw == 1 ? (uint32_t)kWtWords * gw : (uint32_t)kWtWords * gw / 2u);
}

// Queue heads and the error word of the persistent kernels; zeroed before a launch.
struct QueueState {
    unsigned int tile_head;    // tile items
    unsigned int warp_head;    // hash items
    unsigned int cs_head;      // centre-split items (their centre pass)
    unsigned int error;        // nonzero: a kernel saw an impossible state (see kErr*)
    unsigned int wt_head;      // warp-tile items
    unsigned int gt_head;      // group-tile items
};

enum : unsigned int {
    kErrHashFull = 1u,         // a hash table ran out of slots (work estimate was wrong)
    kErrBadItem = 2u,
};

struct Tuning {
    int tile_words;
    int warp_max_wedges;
    int dense_min_permille;
    long long split_wedges;
    int blocks_per_sm;
    int plain;                 // static one-block-per-anchor schedule (Algorithm 3)
    int tiles_only = 0;        // every anchor on block tiles (no hash or warp/group tiles)
    int queue_chunk = 1;       // items per queue access of the warp and group kernels
    int group_warps = 4;       // warps per table of the group-tile kernel (4 or 8)
};

Tuning resolve_tuning(const bbc_tuning *t, int sm_count);

// Motif counts over a graph's tile items (built with tiles_only): kind 1 the six sign
// classes, kind 2 balanced and all (2,k)-bicliques. out (device, 8 words, zeroed by the
// caller): the sums, then an overflow flag in word 7.
bbc_status launch_motif(const DevGraph *graph, const TileItem *items, int n_items, unsigned *head,
                        int kind, int k, int tile_words, int blocks, unsigned long long *out,
                        cudaStream_t st);

// ----------------------------------------------------------------------------- errors

void set_error(const std::string &msg);
bbc_status cuda_fail(cudaError_t e, const char *what);

#define BBC_CUDA_TRY(expr)                                                    \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) return ::bbc::cuda_fail(_e, #expr);            \
    } while (0)

#define BBC_TRY(expr)                                                         \
    do {                                                                      \
        bbc_status _s = (expr);                                               \
        if (_s != BBC_OK) return _s;                                          \
    } while (0)

// ----------------------------------------------------------------------------- accounting

// Every kernel launch of the library bumps a process-wide counter (bbc_launch_count).
void note_launch();

// Optional per-kernel timing (bbc_profile_start / bbc_profile_stop): while enabled, the
// counting kernels are bracketed by CUDA events on their own stream. profile_begin
// returns a token (-1 when profiling is off or the stream is being captured).
enum {
    kProfTile = 0, kProfHash = 1, kProfWarpTile = 2, kProfGroupTile = 3, kProfMotif = 4, kProfTileCs = 5,
    kProfKinds = 6
};
int profile_begin(int kind, cudaStream_t st);
bool profiling_active();
void profile_end(int token, cudaStream_t st);

// ----------------------------------------------------------------------------- memory

// Stream-ordered allocation from the library's own pool on the current device.
bbc_status dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);

template <class T>
bbc_status dev_alloc_n(T **p, size_t n, cudaStream_t st) {
    return dev_alloc(reinterpret_cast<void **>(p), n * sizeof(T) + (n == 0 ? 16 : 0), st);
}

int device_sm_count();
size_t l2_bytes();           // L2 size of the current device
bbc_status check_device();   // the current device is usable (compute capability 10.3)

// ----------------------------------------------------------------------------- sort/scan

// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of the key.
// keys/vals are sorted in place (scratch buffers are allocated from the pool).
bbc_status radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int bits,
                            cudaStream_t st);

// out[i] = sum_{j < i} in[j] for i in [0, n]; out has n + 1 entries.
bbc_status exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n,
                                     cudaStream_t st);
bbc_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t st);
bbc_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st);

// ----------------------------------------------------------------------------- counting

struct CountLaunch {
    const DevGraph *graphs;     // device array
    const TileItem *tile_items; // device
    int32_t n_tile_items;
    const HashItem *warp_items; // device
    int32_t n_warp_items;
    const HashItem *wt_items;   // device, warp-tile items
    int32_t n_wt_items;
    const HashItem *gt_items;   // device, group-tile items
    int32_t n_gt_items;
    QueueState *queue;          // device, zeroed by the caller before the launch
    Tuning tuning;
    long long *item_cycles = nullptr;  // device, per tile item: its duration in SM cycles
    bool prefetch = false;      // the graphs' C -> S rows are larger than L2: the tile kernel
                                // asks for each slice's first lines ahead of use
    // per-vertex counts only: the centre-split items again, for their centre pass after
    // the tile kernel (the graphs' cs_buf and cs_arrive zeroed by the caller)
    const TileItem *cs_items = nullptr;
    int32_t n_cs_items = 0;
    bool per_vertex = false;    // the graphs count per-vertex sums (picks the tile schedule)
};

// One contiguous run of a graph's work items to copy into a combined list, tagged with
// the graph's index in that list's descriptor array.
struct CopyJob {
    const void *src;
    int64_t dst;
    int32_t n;
    int32_t graph;
};

// Copies every job's items (TileItem when `tiles`, else HashItem) into `dst` with one
// kernel; `djobs` is device scratch for jobs.size() entries (the copy of `jobs` into it
// is a pageable host-to-device copy, so `jobs` may be released on return).
bbc_status concat_items(const std::vector<CopyJob> &jobs, bool tiles, void *dst, CopyJob *djobs,
                        cudaStream_t st);

// Queues the counting kernels (block tiles, warp tiles, warp hash) on `st`.
bbc_status launch_count(const CountLaunch &L, cudaStream_t st);
// Creates the calling thread's side streams for launch_count ahead of a stream capture.
bbc_status ensure_side_streams();

// Launches only the tile kernel over `items` with `blocks` persistent blocks; touches no
// memory but the arguments it is given.
bbc_status launch_tile_only(const DevGraph *graphs, const TileItem *items, int n_items,
                            unsigned *head, int tile_words, int blocks, cudaStream_t st);

// Sets the kernels' shared-memory limits on the current device (idempotent); done
// before any stream capture so that capture only records launches.
bbc_status configure_count_kernels();

// Static shared memory of the tile kernel (its dynamic part is the counter tile).
int tile_static_smem_bytes();

// Splits anchors whose wedge count exceeds a fair share of one block's work.
long long auto_split(uint64_t wedges, int sm_count, int blocks_per_sm);

}  // namespace bbc
