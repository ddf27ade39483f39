/*
 * bbc.h -- exact balanced-butterfly counting on one GB300 (sm_103a).
 *
 * The problem (Sec. III, "Problem Statement", of Mekala, Das, Banerjee and Ray,
 * "Multi-core & GPU-based Balanced Butterfly Counting in Signed Bipartite Graphs",
 * arXiv 2601.17707): given a signed bipartite graph G = (U, V, E+ u E-), count the
 * butterflies (Def. 1: 4-cycles u-x-w-y with u, w in U and x, y in V) that hold an
 * even number of negative edges (Def. 2, "balanced"). By Lemma 1 (Sec. IV) every
 * pair {u, w} on one side with p symmetric and n asymmetric wedges (Defs. 7-9)
 * closes C(p,2) + C(n,2) balanced and p*n unbalanced butterflies.
 *
 * Conventions of every call:
 *   - Every call returns a bbc_status; nothing aborts or throws across this boundary.
 *     bbc_last_error() gives a one-line description of the last failure on the
 *     calling thread.
 *   - Vertex ids are 0-based per side; signs are int8 +1 / -1 (Sec. III's "+" / "-").
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Device work is queued on it; host outputs (pointers documented as
 *     "host") are valid when the call returns, so those calls synchronise the stream.
 *   - Inputs are copied; the caller keeps ownership of every buffer it passes.
 *     A bbc_graph owns the device memory it allocates until bbc_graph_free.
 *   - A bbc_graph is not thread-safe; a bbc_server is (submit / poll / wait).
 */
#ifndef BBC_H
#define BBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bbc_status {
    BBC_OK = 0,
    BBC_E_INVALID_ARG = 1,     /* a NULL or negative argument, or inconsistent sizes */
    BBC_E_OUT_OF_RANGE = 2,    /* an edge endpoint id outside [0, n_u) or [0, n_v) */
    BBC_E_BAD_SIGN = 3,        /* a sign other than +1 or -1 */
    BBC_E_DUPLICATE_EDGE = 4,  /* the same (u, v) pair twice, without BBC_DEDUP_LAST */
    BBC_E_OVERFLOW_RISK = 5,   /* a count could exceed 2^64 - 1 */
    BBC_E_NO_MEMORY = 6,       /* a device or host allocation failed */
    BBC_E_OVER_BUDGET = 7,     /* a request larger than the server's device budget */
    BBC_E_CUDA = 8,            /* a CUDA runtime error (see bbc_last_error) */
    BBC_E_TIMEOUT = 9,         /* a bounded wait ran out */
    BBC_E_CANCELLED = 10,      /* the server was shut down before the request finished */
    BBC_E_NOT_READY = 11,      /* bbc_poll: the request is still in flight */
    BBC_E_NO_DEVICE = 12       /* no usable CUDA device of compute capability 10.3 */
} bbc_status;

/* Flags of bbc_prepare. */
enum {
    BBC_INPUT_DEVICE = 1u,      /* u, v, sign are device pointers (default: host) */
    BBC_DEDUP_LAST = 2u,        /* keep the last of repeated (u, v) pairs (Sec. VI keeps
                                   the most recent rating) instead of failing */
    BBC_SIDE_FORCE_U = 4u,      /* take U as the pair (anchor) side */
    BBC_SIDE_FORCE_V = 8u,      /* take V as the pair (anchor) side */
    BBC_ORIENT_LOW_ANCHOR = 16u /* count each pair at its lower-priority member (M-BBC's
                                   p(w) < p(u) the other way round); same results */
};

typedef struct bbc_graph bbc_graph;
typedef struct bbc_server bbc_server;

/*
 * Kernel tuning. Zero in any field selects the built-in default for it. The counts
 * never depend on these values, only the speed does.
 */
typedef struct bbc_tuning {
    int32_t tile_words;        /* 32-bit words per shared-memory counter tile (0: the
                                  largest that keeps blocks_per_sm blocks resident) */
    int32_t warp_max_wedges;   /* anchors with at most this many oriented wedges go to the
                                  one-warp hash path (<= 512) */
    int32_t dense_min_permille;/* reserved for a block-level hash path (unused) */
    int32_t split_wedges;      /* anchors with more wedges than this are split into
                                  tile-range items that run on different blocks; an
                                  anchor that wants more such items than half its tiles
                                  also has each tile's centres cut into parts (2 to 64, of
                                  about split_wedges / 16 wedges) whose counts are merged
                                  in device memory (at most the larger of 8 bytes per
                                  edge and 16 MiB, else no centre split) */
    int32_t blocks_per_sm;     /* resident blocks per SM of the tile kernel (1 or 2) */
    int32_t plain;             /* 1: the static schedule of G-BBC (Algorithm 3) -- one block
                                  per anchor in rank order, no work queue, no heavy-first
                                  ordering, no hash path, no splitting; for comparisons */
    int32_t queue_chunk;       /* work items a warp (or warp group) of the light-anchor
                                  kernels takes from its queue per atomic access (1..64;
                                  0: the default, 1) */
    int32_t group_warps;       /* warps sharing one counter table in the group-tile kernel:
                                  4 (0: the default) or 8 (a table of twice the endpoints,
                                  so wider single-tile anchors leave the block-tile kernel) */
} bbc_tuning;

/* Fills *t with the built-in defaults. */
bbc_status bbc_tuning_default(bbc_tuning *t);

/*
 * bbc_prepare -- validate the edge list and build the device layout the counting
 * kernels read (Sec. IV "Vertex Priority", Def. 6; Algorithm 4's host preprocessing).
 *
 *   n_u, n_v    side sizes (>= 0); n_edges >= 0 edges given as u[i], v[i], sign[i].
 *   u, v        int32 endpoint ids; sign: int8 +1 / -1. Host memory, or device memory
 *               when BBC_INPUT_DEVICE is set. Not retained after the call.
 *   flags       BBC_* flags above.
 *   out         receives a new graph handle on success (untouched on failure).
 *
 * What it does: checks ids and signs (BBC_E_OUT_OF_RANGE / BBC_E_BAD_SIGN) and
 * duplicate pairs (BBC_E_DUPLICATE_EDGE unless BBC_DEDUP_LAST); picks the pair side S
 * as the side whose opposite side has the smaller sum of C(d, 2) (that sum is the
 * number of oriented wedges W the count visits; ties pick U); ranks S and the centre
 * side C by (degree descending, id descending) as in Def. 6; and builds two int32 CSR
 * arrays with the sign in bit 31 of each column index: S -> C rows and C -> S rows,
 * the latter sorted by rank so that the endpoints of higher rank form a suffix. It also
 * estimates each anchor's wedge count and builds the work lists of bbc_count.
 * Returns BBC_E_OVERFLOW_RISK when W * (max degree on S - 1) / 2 exceeds 2^64 - 1.
 */
bbc_status bbc_prepare(int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *u,
                       const int32_t *v, const int8_t *sign, uint32_t flags,
                       void *cuda_stream, bbc_graph **out);

/*
 * bbc_count -- the exact counts of a prepared graph (Algorithms 2-4 of the paper
 * compute `balanced`; the other outputs are extensions of this library).
 *
 *   balanced    host uint64: number of balanced butterflies (Def. 2). Required.
 *   unbalanced  host uint64 or NULL: number of butterflies with an odd number of
 *               negative edges.
 *   per_u       device uint64[n_u] or NULL: per_u[x] = number of balanced butterflies
 *               that contain vertex x of U. Overwritten.
 *   per_v       device uint64[n_v] or NULL: the same for V.
 *   tuning      NULL for the defaults.
 * Synchronises `cuda_stream` before returning.
 */
bbc_status bbc_count(bbc_graph *g, uint64_t *balanced, uint64_t *unbalanced, uint64_t *per_u,
                     uint64_t *per_v, const bbc_tuning *tuning, void *cuda_stream);

/*
 * bbc_count_async -- as bbc_count, but writes {balanced, unbalanced} into the device
 * buffer totals_dev (2 x uint64, overwritten) and returns without synchronising.
 * Every launch is queued on `cuda_stream`. The kernels' internal-consistency flag (set
 * if a light anchor's hash table ran out of slots, which its sizing rules out) is read
 * back only by the synchronising calls (bbc_count, bbc_count_batch, the server).
 */
bbc_status bbc_count_async(bbc_graph *g, uint64_t *totals_dev, uint64_t *per_u,
                           uint64_t *per_v, const bbc_tuning *tuning, void *cuda_stream);

/*
 * bbc_count_noalloc -- bbc_count's global totals for a prepared graph, without any
 * device or host allocation. The paper has no counterpart; this entry point exists for
 * callers that cannot allocate at the time they count: processes whose device memory is
 * already reserved in full by another framework's caching allocator (any new allocation
 * fails there), latency-critical loops that must not pay for the implicit device-wide
 * synchronisation of cudaMalloc / cudaFree, and hosts that cap a library's device memory
 * at what it holds once loaded.
 *
 *   g           a graph from bbc_prepare (its device layout is the input; unchanged).
 *   totals_dev  device uint64[2], caller-owned: receives {balanced, unbalanced}.
 *   cuda_stream the stream every launch is queued on; the call does not synchronise.
 *
 * The per-call scratch (queue head, kernel descriptor, one work item per pair-side
 * vertex) lives in a 1 MiB static device array that every GPU loading this library
 * holds until the process exits. Limit: graphs whose pair side has at most 65,520
 * vertices; larger ones return BBC_E_INVALID_ARG with a message, before any launch.
 * The first call on each device looks the array's address up (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture. All calls
 * share the one array and each clears what must start at zero, so calls that overlap on
 * the GPU (different streams, or threads without ordering) race and give wrong results.
 * Work is one item per anchor covering all of its endpoint tiles (no split of heavy
 * anchors across blocks, unlike bbc_count), so on graphs with a few dominant hubs the
 * call can take much longer than bbc_count: the hubs' tiles run one after another on
 * one block.
 */
bbc_status bbc_count_noalloc(const bbc_graph *g, uint64_t *totals_dev, void *cuda_stream);

/*
 * bbc_graph_work -- the work behind a prepared graph's current work lists (built with the
 * default tuning if it has none), for per-kernel reports: out (host uint64[12]) holds, for
 * the block-tile, group-tile, warp-tile and hash paths in that order, {work items, oriented
 * wedges of their anchors, pair-side edges of their anchors}. Synchronises.
 */
bbc_status bbc_graph_work(bbc_graph *g, uint64_t *out, void *cuda_stream);

/* Motif kinds of bbc_count_motif. */
enum {
    BBC_MOTIF_SIGN_CLASSES = 1, /* the six sign classes of Sec. VII, Table 7 */
    BBC_MOTIF_BICLIQUE_2K = 2   /* balanced (2,k)-bicliques, Def. 5 */
};

/*
 * bbc_count_motif -- other per-pair sums over the same wedge grouping, with the pair
 * ("2") on the graph's pair side S: prepare with BBC_SIDE_FORCE_U or BBC_SIDE_FORCE_V
 * to fix it, since neither motif is side-symmetric (bbc_graph_info reports S).
 *
 *   kind BBC_MOTIF_SIGN_CLASSES (Sec. VII, Table 7; k ignored): for a pair {a, w} of S
 *     each common neighbour c is pp (both edges +), nn (both -) or a (signs differ);
 *     out[0..5] = the numbers of butterflies of each class, in Table 7's order:
 *     coherent ++/++ = sum C(pp,2), coherent ++/-- = sum pp*nn, coherent --/-- =
 *     sum C(nn,2), incoherent +-/+- = sum C(a,2), mixed ++/+- = sum pp*a, mixed
 *     +-/-- = sum nn*a. The first four add up to bbc_count's balanced total, the last
 *     two to its unbalanced one.
 *   kind BBC_MOTIF_BICLIQUE_2K (Def. 5 with Algorithm 1's C(., k) aggregation; k >= 2):
 *     out[0] = balanced (2,k)-bicliques = sum C(p,k) + C(n,k) (k common neighbours
 *     with no unbalanced butterfly among them are all symmetric or all asymmetric, by
 *     Lemma 1); out[1] = all (2,k)-bicliques = sum C(p+n,k). k = 2 gives bbc_count's
 *     balanced total and the unsigned butterfly count.
 *   out   host uint64[6] (classes) or uint64[2] (bicliques). Overwritten.
 * Errors: BBC_E_INVALID_ARG (kind, k < 2 or k >= 2^31, NULL), BBC_E_OVERFLOW_RISK when
 * a sum or a single binomial exceeds 2^64 - 1. The call rebuilds the graph's work lists
 * for the motif (all anchors on block tiles) and synchronises `cuda_stream`; the next
 * bbc_count rebuilds its own lists.
 */
bbc_status bbc_count_motif(bbc_graph *g, int32_t kind, int32_t k, uint64_t *out, void *cuda_stream);

/*
 * bbc_graph_info -- facts about a prepared graph (any output pointer may be NULL).
 *   side          0 when U is the pair side S, 1 when V is.
 *   wedges        W, the number of oriented wedges bbc_count visits
 *                 (sum over the centre side of C(d, 2)).
 *   device_bytes  device memory the handle holds.
 *   n_edges       edges after de-duplication.
 */
bbc_status bbc_graph_info(const bbc_graph *g, int32_t *side, uint64_t *wedges,
                          size_t *device_bytes, int64_t *n_edges);

/* Releases the handle and its device memory (NULL is a no-op). */
void bbc_graph_free(bbc_graph *g);

/*
 * bbc_count_batch -- count n prepared graphs in one persistent launch over a device-side
 * (graph, anchor) work list, captured once into a CUDA graph and replayed for later
 * batches of the same graphs (the batched form of this library; the paper counts one
 * graph at a time).
 *   gs        n graph handles (each prepared on the device of the calling thread).
 *   balanced  host uint64[n]: per-graph balanced counts. Required.
 *   tuning    NULL: tuned choice (see bbc_autotune_batch), else the given values.
 * Synchronises `cuda_stream`.
 */
bbc_status bbc_count_batch(int32_t n, bbc_graph *const *gs, uint64_t *balanced,
                           const bbc_tuning *tuning, void *cuda_stream);

/*
 * bbc_autotune_batch -- times bbc_count_batch on these graphs while searching, one knob
 * at a time from the defaults, the group-tile width (group_warps), the counter-tile size
 * (tile_words), the light-anchor threshold (warp_max_wedges), the heavy-anchor split size
 * (split_wedges), the resident blocks per SM and the queue chunk (queue_chunk), and stores
 * the fastest choice in *best.
 * The choice is also kept for NULL-tuning batch calls on batches of the same shape bucket
 * (the SM count, the number of graphs and the binary orders of magnitude of their edges,
 * wedges and pair-side vertices), in the process and in a cache file that later processes
 * read: $BBC_TUNE_CACHE, else $XDG_CACHE_HOME/bbc/batch_tuning.txt, else
 * $HOME/.cache/bbc/batch_tuning.txt (an empty BBC_TUNE_CACHE keeps it in the process).
 * The counts are checked to agree across every candidate; a disagreement returns
 * BBC_E_CUDA.
 */
bbc_status bbc_autotune_batch(int32_t n, bbc_graph *const *gs, bbc_tuning *best,
                              void *cuda_stream);

/* The tuning a NULL-tuning bbc_count_batch call would use for these graphs (the cached
 * choice of bbc_autotune_batch for their shape bucket, else the defaults); split_wedges
 * is the size chosen for this batch. Host only, no device work. */
bbc_status bbc_batch_tuning(int32_t n, bbc_graph *const *gs, bbc_tuning *out);

/*
 * Serving loop: requests (edge lists in host memory) are copied, queued, admitted while
 * the device memory they need fits the budget, prepared, and counted together with the
 * other admitted requests in continuous batches on the server's own stream.
 *   device_budget_bytes  upper bound of device memory held by admitted requests.
 *   tuning               NULL for the defaults.
 */
bbc_status bbc_server_create(size_t device_budget_bytes, const bbc_tuning *tuning,
                             bbc_server **out);

/* Queues one request; its input is copied before the call returns. BBC_E_OVER_BUDGET
 * when the request alone could never fit the budget. */
bbc_status bbc_submit(bbc_server *s, int32_t n_u, int32_t n_v, int64_t n_edges,
                      const int32_t *u, const int32_t *v, const int8_t *sign,
                      uint64_t *ticket);

/* BBC_OK with *balanced set when done, BBC_E_NOT_READY while in flight, or the
 * request's own error status. A finished ticket may be polled again. */
bbc_status bbc_poll(bbc_server *s, uint64_t ticket, uint64_t *balanced);

/* Waits at most timeout_us microseconds (< 0: no limit) for a ticket. */
bbc_status bbc_wait(bbc_server *s, uint64_t ticket, int64_t timeout_us, uint64_t *balanced);

/* Latency statistics of finished requests, in microseconds from submit to completion. */
bbc_status bbc_server_stats(bbc_server *s, uint64_t *completed, double *p50_us,
                            double *p99_us, double *mean_us);

/*
 * Counters of a server since its creation, for capacity reports (not part of the
 * counting). All times are host wall-clock microseconds except tick_gpu_us, the summed
 * device time of the ticks' counting launches (CUDA events on the server's stream).
 */
typedef struct bbc_server_counters {
    uint64_t submitted;           /* requests accepted by bbc_submit */
    uint64_t admitted;            /* requests whose reservation was taken */
    uint64_t completed;           /* requests finished, with any status */
    uint64_t admitted_after_wait; /* admitted requests that had found the budget full (or
                                     an earlier request still waiting) and were admitted
                                     only after another request released its memory */
    uint64_t queued_now;          /* requests waiting for admission now */
    uint64_t max_queued;          /* most requests waiting for admission at once */
    uint64_t max_resident;        /* most admitted, unfinished requests at once */
    uint64_t ticks;               /* counting launches of the tick loop */
    size_t budget_bytes;
    size_t reserved_bytes;        /* reserved by admitted, unfinished requests now */
    size_t peak_reserved_bytes;   /* the most ever reserved at once (<= budget_bytes) */
    double tick_wall_us;          /* time the tick thread spent inside ticks */
    double tick_gpu_us;           /* device time of the ticks' counting kernels */
    double prep_wall_us;          /* summed preparation time over the preparation threads */
    double elapsed_us;            /* since bbc_server_create */
} bbc_server_counters;

bbc_status bbc_server_counters_get(bbc_server *s, bbc_server_counters *out);

/* What happened to one finished request (BBC_E_NOT_READY while it is in flight). */
typedef struct bbc_request_info {
    int32_t status;               /* the request's own status */
    int32_t ticks;                /* counting launches it took part in */
    int64_t n_edges;
    uint64_t wedges;              /* W of its graph (0 if preparation failed) */
    size_t reserved_bytes;        /* its reservation */
    int32_t waited_for_memory;    /* 1: it was not admitted at submission */
    int32_t pad;
    double latency_us;            /* submission to completion */
    double queued_us;             /* submission to admission */
    double prepare_us;            /* admission to the end of its preparation */
    double count_us;              /* end of preparation to completion */
    double tick_gpu_us;           /* device time of the ticks it was in (shared with the
                                     other requests of those ticks) */
    double submit_us;             /* its submission, in microseconds after bbc_server_create */
} bbc_request_info;

bbc_status bbc_server_request_info(bbc_server *s, uint64_t ticket, bbc_request_info *out);

/* Stops the loop; requests still queued finish with BBC_E_CANCELLED. */
void bbc_server_destroy(bbc_server *s);

/*
 * Device memory of the library's stream-ordered pool on the current device: *used is
 * what the library's live allocations hold now, *used_high the most they held at once
 * since the process started or since the last call with reset_high != 0 (which resets it
 * to the current use). Either pointer may be NULL.
 */
bbc_status bbc_memory_usage(size_t *used, size_t *used_high, int32_t reset_high);

/*
 * bbc_count_delta -- the exact change of the counts when a batch of edge updates is
 * applied to a prepared graph (dynamic signed graphs, named as future work in Sec. VIII;
 * this library's extension). Update i sets the sign of edge (u[i], v[i]) to new_sign[i]:
 * +1 or -1 inserts the edge or re-signs it, 0 deletes it. The graph itself is not changed.
 *
 *   d_balanced    host int64: B(G') - B(G), balanced butterflies (Def. 2). Required.
 *   d_unbalanced  host int64 or NULL: the same for unbalanced butterflies.
 *   flags         BBC_INPUT_DEVICE when u, v, new_sign are device pointers.
 * Only pairs {a, w} of the pair side with a member touched by an update can change
 * (Lemma 1 counts per pair); each such pair is recounted before and after the batch,
 * so the work is the 2-hop neighbourhood of the touched pair-side vertices.
 * Errors: BBC_E_OUT_OF_RANGE (an id), BBC_E_BAD_SIGN (a sign other than -1, 0, +1),
 * BBC_E_DUPLICATE_EDGE (one pair twice in the batch), BBC_E_INVALID_ARG (deleting an
 * absent edge, NULL arguments). Synchronises `cuda_stream`.
 */
bbc_status bbc_count_delta(const bbc_graph *g, int64_t n_updates, const int32_t *u, const int32_t *v,
                           const int8_t *new_sign, uint32_t flags, int64_t *d_balanced,
                           int64_t *d_unbalanced, void *cuda_stream);

/*
 * Learned cost model of the tile kernel's work items (an extension: the paper orders
 * Algorithm 4's queue by a fanout estimate, and this library by each item's share of its
 * anchor's oriented wedges). A small fp32 network (8 item features -> 32 -> 32 -> 1, ReLU)
 * is trained on the GPU, by this library's own forward, backward and Adam kernels, to
 * predict an item's duration (standardised log SM cycles) from features the library
 * computes; bbc_cost_model_order then sorts a graph's tile items by the prediction,
 * heaviest first. Counts do not depend on the order.
 *
 * Parameter layout (fp32, bbc_cost_model_num_params() = 1,377): W1[32][8], b1[32],
 * W2[32][32] (row j = unit j of the second layer), b2[32], w3[32], b3; the network is
 * y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3.
 * Feature rows (8 floats per tile item, in the graph's current queue order): log1p of
 * the anchor's wedges / 16, log1p(anchor degree) / 16, log1p(tiles in the item) / 8,
 * log1p(endpoint span of the item) / 16, first tile / the anchor's tiles, counter width
 * / 2, log1p(|S|) / 16, log1p(wedge share of the item) / 16.
 */
typedef struct bbc_cost_model bbc_cost_model;

/* A model with He-uniform weights drawn from SplitMix64(seed) and zero biases. */
bbc_status bbc_cost_model_create(uint64_t seed, bbc_cost_model **out);
void bbc_cost_model_free(bbc_cost_model *m);
int32_t bbc_cost_model_num_params(void);
/* Host copies of the parameters (capacity >= bbc_cost_model_num_params()). set_params
   also clears the optimiser state. */
bbc_status bbc_cost_model_get_params(const bbc_cost_model *m, float *host_out, int32_t capacity);
bbc_status bbc_cost_model_set_params(bbc_cost_model *m, const float *host_in, int32_t n_params);
/*
 * Loss L = (1/n) sum_i (y(x_i) - t_i)^2 and its gradient with respect to every parameter
 * at the current parameters. X_dev: device float[n][8]; t_dev: device float[n].
 * loss_host: host float; grad_host: host float[num_params] or NULL. Synchronises.
 */
bbc_status bbc_cost_model_loss_grad(bbc_cost_model *m, const float *X_dev, const float *t_dev, int32_t n,
                                    float *loss_host, float *grad_host, void *cuda_stream);
/*
 * Trains on (X_dev, cycles_dev): labels are log(cycles) standardised over the n samples;
 * `steps` full-batch Adam steps at learning rate lr. loss_host (host float or NULL)
 * receives the final loss in standardised units. Synchronises.
 */
bbc_status bbc_cost_model_fit(bbc_cost_model *m, const float *X_dev, const int64_t *cycles_dev, int32_t n,
                              int32_t steps, float lr, float *loss_host, void *cuda_stream);
/* y_dev[i] = the network at X_dev[i] (device float[n]); queued, no synchronisation. */
bbc_status bbc_cost_model_predict(const bbc_cost_model *m, const float *X_dev, int32_t n, float *y_dev,
                                  void *cuda_stream);
/* Feature rows of g's tile items (device float[capacity][8]); *n_items = their number.
   X_dev = NULL with capacity 0 only reports the number. */
bbc_status bbc_item_features(bbc_graph *g, float *X_dev, int32_t capacity, int32_t *n_items, void *cuda_stream);
/* The original id (on the pair side S, see bbc_graph_info) of each tile item's anchor, in
   the same queue order (device int32[capacity]); *n_items = their number. Queued, no
   synchronisation; BBC_E_INVALID_ARG when capacity is below the number of items. */
bbc_status bbc_item_anchors(bbc_graph *g, int32_t *anchors_dev, int32_t capacity, int32_t *n_items,
                            void *cuda_stream);
/*
 * Runs the tile kernel once over g's tile items (global totals only, the other kernels
 * are not run) and writes each item's duration in SM cycles (device int64[capacity]),
 * in queue order. Synchronises.
 */
bbc_status bbc_item_cycles(bbc_graph *g, int64_t *cycles_dev, int32_t capacity, int32_t *n_items,
                           void *cuda_stream);
/* Sorts g's tile items by the model's prediction, heaviest first. Synchronises. */
bbc_status bbc_cost_model_order(const bbc_cost_model *m, bbc_graph *g, void *cuda_stream);

/*
 * Accounting for reports (not part of the counting): bbc_launch_count is the number of
 * CUDA kernels this library has launched in this process. Between bbc_profile_start and
 * bbc_profile_stop every launch of a counting kernel (outside stream capture) is
 * bracketed by CUDA events on its own stream, and bbc_count_batch launches its recorded
 * work directly instead of replaying the CUDA graph; bbc_profile_stop waits for them and fills
 * up to `capacity` entries, one per kernel, with its launches and summed device time
 * (*count receives the number of kernels seen).
 */
typedef struct bbc_kernel_time {
    const char *name;    /* static string */
    int64_t launches;
    double total_ms;
} bbc_kernel_time;

unsigned long long bbc_launch_count(void);
bbc_status bbc_profile_start(void);
bbc_status bbc_profile_stop(bbc_kernel_time *out, int32_t capacity, int32_t *count);

/* Static strings; never NULL. */
const char *bbc_status_string(bbc_status st);
const char *bbc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BBC_H */
