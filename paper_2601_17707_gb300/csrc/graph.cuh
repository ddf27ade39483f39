// graph.cuh -- the host-side handle of a prepared graph (the opaque bbc_graph of bbc.h).
#pragma once

#include "bbc_internal.cuh"

struct bbc_graph {
    uint64_t uid = 0;          // unique per handle within the process (never reused)
    int device = 0;
    int32_t n_u = 0, n_v = 0;
    int64_t n_edges = 0;       // after de-duplication
    int side = 0;              // 0: S = U (pairs on U, centres on V); 1: S = V
    int side_paper_rule = 0;   // the paper's choice S = min(|U|, |V|) (Alg. 2-4), for reports
    int orient_low = 0;
    int32_t nS = 0, nC = 0;
    uint64_t wedges = 0;       // W = sum over C of C(d, 2)
    int32_t max_deg_S = 0, max_deg_C = 0;

    // device layout (owned)
    int64_t *rowS_off = nullptr;
    uint32_t *rowS = nullptr;
    int64_t *rowC_off = nullptr;
    uint32_t *rowC = nullptr;
    int32_t *permS = nullptr;  // rank -> original id
    int32_t *permC = nullptr;
    unsigned long long *wl = nullptr;  // oriented wedges per anchor rank
    uint2 *rng = nullptr;      // per S -> C entry (a, c): a's endpoint range [x, y) in rowC
    uint32_t *anchor_of = nullptr;  // per S -> C entry: its anchor's rank
    uint32_t *bnd = nullptr;   // interior tile boundaries for the current work lists
    int64_t *boff = nullptr;   // nS + 1 offsets into bnd
    uint64_t layout_version = 0;    // bumped whenever the work lists are rebuilt

    // work lists (rebuilt when the tuning changes)
    bbc::Tuning items_tuning{};
    bool items_valid = false;
    bbc::TileItem *tile_items = nullptr;
    int32_t n_tile = 0;
    bbc::HashItem *warp_items = nullptr;
    int32_t n_warp = 0;
    bbc::HashItem *wt_items = nullptr;
    int32_t n_wt = 0;
    bbc::HashItem *gt_items = nullptr;
    int32_t n_gt = 0;
    // centre-split tiles: per item its record, the items again (their centre pass), and
    // per tile group the merged counters and an arrival counter
    bbc::CentreSplit *cs_desc = nullptr;
    bbc::TileItem *cs_items = nullptr;
    int32_t n_cs_items = 0;
    uint32_t *cs_buf = nullptr;
    unsigned *cs_arrive = nullptr;
    int64_t n_cs_groups = 0;
    int64_t cs_group_words = 0;

    // count-time state
    bbc::DevGraph *dgraph = nullptr;       // device copy of the descriptor
    unsigned long long *bS = nullptr;      // per-vertex by rank, allocated on first use
    unsigned long long *bC = nullptr;
    unsigned long long *totals = nullptr;  // 2 words
    bbc::QueueState *queue = nullptr;

    size_t device_bytes = 0;
};

namespace bbc {

bbc_status prepare_graph(int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *u,
                         const int32_t *v, const int8_t *sign, uint32_t flags, cudaStream_t st,
                         bbc_graph **out);
bbc_status build_work_lists(bbc_graph *g, const Tuning &t, cudaStream_t st);
void release_graph(bbc_graph *g, cudaStream_t st);
// The kernels' view of g. with_bounds: the tile boundaries of the work lists last
// built (pass true only right after build_work_lists with the tuning being launched).
DevGraph host_descriptor(const bbc_graph *g, bool per_vertex, bool with_bounds = false);
// The graph's C -> S rows (4 bytes per edge) are larger than the device's L2.
bool rows_exceed_l2(const bbc_graph *g);
// Zeroes the merged counters and arrival counters of g's centre-split tiles (queued on
// st); every launch of the tile kernel over g's items needs it first.
bbc_status clear_centre_split(const bbc_graph *g, cudaStream_t st);

}  // namespace bbc
