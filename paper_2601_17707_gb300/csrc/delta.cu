// delta.cu -- exact count changes of a batch of edge updates (dynamic signed graphs).
//
// The paper names dynamic signed bipartite graphs (edges added, removed, or re-signed)
// as future work (Sec. VIII). Here a batch D of updates on a prepared graph G gives
// G', and the call returns B(G') - B(G) and the same for unbalanced butterflies without
// recounting G'. By Lemma 1 the counts are sums over pairs {a, w} of the pair side S of
// f(p, n) = C(p,2) + C(n,2) (and p * n), where p and n count the common neighbours
// reached by symmetric and asymmetric wedges. A pair's (p, n) changes only through an
// edge (a, c) or (w, c) in D, so only pairs with a member in A, the set of S vertices that
// an update touches, can change. For every a in A the pair vector of a is recounted in G
// and in G' (all endpoints w, no orientation), one endpoint tile per block at a time, and
// each pair {a, w} adds f(G') - f(G) once: at a when w is outside A or ranks above a.
//
// Steps: ids -> ranks (k_rank_of); updates -> (a, c, old sign from the CSR, new sign)
// with range and sign checks (k_map_updates); stable radix sorts by a and by (c, a);
// duplicate and absent-deletion checks (k_check_updates); the distinct anchors A
// (k_anchor_marks + scan); work items (anchor, endpoint tile), heaviest anchors first
// (k_delta_plan, a radix sort, a scan); persistent blocks over the items (k_delta_tile),
// each with a shared-memory tile of four counters per endpoint (old p, old n, new p,
// new n) that the anchor's centre rows fill and the tile's epilogue turns into changes.
#include "graph.cuh"

namespace bbc {
namespace {

constexpr int kDeltaThreads = 256;
constexpr int kDeltaWarps = kDeltaThreads / 32;
constexpr uint32_t kAbsent = 0;   // sign code: 0 absent, 1 positive, 2 negative

enum : unsigned { kErrRange = 1u, kErrSign = 2u, kErrDup = 4u, kErrAbsent = 8u };

__global__ void k_rank_of(const int32_t *__restrict__ perm, int64_t n, int32_t *__restrict__ rank) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        rank[perm[r]] = (int32_t)r;
}

// The sign code of edge (a, c) in G: binary search of anchor rank a in the C -> S row of
// c (those rows are sorted by rank; the S -> C rows keep input order).
__device__ uint32_t old_code(const int64_t *__restrict__ rowC_off, const uint32_t *__restrict__ rowC,
                             uint32_t a, uint32_t c) {
    int64_t lo = rowC_off[c], hi = rowC_off[c + 1];
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        const uint32_t x = rowC[m] & kIdMask;
        if (x < a)
            lo = m + 1;
        else
            hi = m;
    }
    if (lo < rowC_off[c + 1] && (rowC[lo] & kIdMask) == a) return (rowC[lo] >> 31) ? 2u : 1u;
    return kAbsent;
}

// Per update i: anchor rank a, centre rank c, old and new sign codes.
__global__ void k_map_updates(const int32_t *__restrict__ u, const int32_t *__restrict__ v,
                              const int8_t *__restrict__ s, int64_t n, int32_t n_u, int32_t n_v, int side,
                              const int32_t *__restrict__ rankS, const int32_t *__restrict__ rankC,
                              const int64_t *__restrict__ rowC_off, const uint32_t *__restrict__ rowC,
                              uint32_t *__restrict__ ua, uint32_t *__restrict__ uc, uint8_t *__restrict__ uold,
                              uint8_t *__restrict__ unew, unsigned *__restrict__ err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = u[i], y = v[i];
        const int8_t sg = s[i];
        if (x < 0 || x >= n_u || y < 0 || y >= n_v) {
            atomicOr(err, kErrRange);
            ua[i] = uc[i] = 0;
            uold[i] = unew[i] = 0;
            continue;
        }
        if (sg != 1 && sg != -1 && sg != 0) atomicOr(err, kErrSign);
        const uint32_t a = (uint32_t)(side == 0 ? rankS[x] : rankS[y]);
        const uint32_t c = (uint32_t)(side == 0 ? rankC[y] : rankC[x]);
        ua[i] = a;
        uc[i] = c;
        uold[i] = (uint8_t)old_code(rowC_off, rowC, a, c);
        unew[i] = (uint8_t)(sg == 1 ? 1 : (sg == -1 ? 2 : 0));
    }
}

__global__ void k_iota_u32(uint32_t *__restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (uint32_t)i;
}

__global__ void k_gather_u8(const uint8_t *__restrict__ src, const uint32_t *__restrict__ order, int64_t n,
                            uint8_t *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[order[i]];
}

__global__ void k_gather_u32(const uint32_t *__restrict__ src, const uint32_t *__restrict__ order, int64_t n,
                             uint32_t *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[order[i]];
}

// In (c, a) order: keys (c << 32 | a) and codes; rejects repeated pairs and deletions of
// absent edges.
__global__ void k_check_updates(const uint32_t *__restrict__ order, const uint32_t *__restrict__ ua,
                                const uint32_t *__restrict__ uc, const uint8_t *__restrict__ uold,
                                const uint8_t *__restrict__ unew, int64_t n, unsigned long long *__restrict__ key,
                                uint8_t *__restrict__ kold, uint8_t *__restrict__ knew, unsigned *__restrict__ err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = order[i];
        key[i] = ((unsigned long long)uc[j] << 32) | ua[j];
        kold[i] = uold[j];
        knew[i] = unew[j];
        if (uold[j] == kAbsent && unew[j] == kAbsent) atomicOr(err, kErrAbsent);
        if (i > 0) {
            const uint32_t p = order[i - 1];
            if (uc[p] == uc[j] && ua[p] == ua[j]) atomicOr(err, kErrDup);
        }
    }
}

// Marks the first update of every distinct anchor in a-sorted order.
__global__ void k_anchor_marks(const uint32_t *__restrict__ a_sorted, int64_t n, int32_t *__restrict__ first,
                               uint8_t *__restrict__ in_a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool f = i == 0 || a_sorted[i] != a_sorted[i - 1];
        first[i] = f ? 1 : 0;
        if (f) in_a[a_sorted[i]] = 1;
    }
}

__global__ void k_anchor_list(const uint32_t *__restrict__ a_sorted, const int32_t *__restrict__ first,
                              const int64_t *__restrict__ pos, int64_t n, uint32_t *__restrict__ anchors,
                              uint32_t *__restrict__ seg_begin) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (first[i]) {
            anchors[pos[i]] = a_sorted[i];
            seg_begin[pos[i]] = (uint32_t)i;
        }
}

// The first index in the (c, a)-sorted keys that is >= k.
__device__ __forceinline__ int64_t lower_key(const unsigned long long *__restrict__ key, int64_t n,
                                             unsigned long long k) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (key[m] < k)
            lo = m + 1;
        else
            hi = m;
    }
    return lo;
}

struct DeltaArgs {
    const int64_t *rowS_off;
    const uint32_t *rowS;
    const int64_t *rowC_off;
    const uint32_t *rowC;
    int64_t nS;
    // updates in (c, a) order
    const unsigned long long *key;
    const uint8_t *kold, *knew;
    int64_t n_upd;
    // updates in a order (centre and codes), with the distinct anchors and their segments
    const uint32_t *c_by_a;
    const uint8_t *old_by_a, *new_by_a;
    const uint32_t *anchors, *seg_begin;
    int32_t n_anchors;
    const uint8_t *in_a;
    // work items: anchor k (in the order `order`) owns items toff[k] .. toff[k + 1] - 1,
    // one per endpoint tile; cw[k] is its counter width code
    const uint32_t *order;
    const int64_t *toff;
    const uint8_t *cw;
    int64_t n_items;
    int32_t tile_words;
    unsigned *next_item;
    unsigned long long *out;   // [0] delta balanced, [1] delta unbalanced (two's complement)
};

// The new sign code of edge (a, c) given its old one.
__device__ __forceinline__ uint32_t new_code(const DeltaArgs &A, uint32_t a, uint32_t c, uint32_t oa) {
    const unsigned long long k = ((unsigned long long)c << 32) | a;
    const int64_t q = lower_key(A.key, A.n_upd, k);
    return (q < A.n_upd && A.key[q] == k) ? A.knew[q] : oa;
}

// First index of row[b, e) whose rank is >= key.
__device__ __forceinline__ int64_t lower_rank(const uint32_t *__restrict__ row, int64_t b, int64_t e, uint32_t key) {
    while (b < e) {
        const int64_t m = (b + e) >> 1;
        if ((row[m] & kIdMask) < key)
            b = m + 1;
        else
            e = m;
    }
    return b;
}

// Anchor k's counter width: a pair's old or new count is at most the anchor's number of
// centres before or after the batch.
__global__ void k_delta_plan(DeltaArgs A, const uint32_t *__restrict__ seg_end, int32_t *__restrict__ ntiles,
                             uint8_t *__restrict__ cw, uint32_t *__restrict__ deg_key) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < A.n_anchors;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = A.anchors[k];
        const int64_t deg = A.rowS_off[a + 1] - A.rowS_off[a];
        const int64_t bound = deg + (int64_t)(seg_end[k] - A.seg_begin[k]);
        const int w = bound <= 255 ? 0 : (bound <= 65535 ? 1 : 2);
        const int64_t ept = (int64_t)A.tile_words >> w;   // 1, 2 or 4 words per endpoint
        cw[k] = (uint8_t)w;
        ntiles[k] = (int32_t)((A.nS + ept - 1) / ept);
        // heaviest anchors first: the sort key is the complement of the degree
        deg_key[k] = 0xffffffffu - (uint32_t)(bound < 0xffffffffll ? bound : 0xffffffffll);
    }
}

constexpr int kDeltaTileThreads = 512;
constexpr int kDeltaTileWarps = kDeltaTileThreads / 32;

// Per chunk of up to 512 centres of an item's anchor: the slice of each centre's row in
// the item's endpoint tile, its old / new anchor-edge codes and its range of updates.
struct DeltaChunk {
    uint32_t c[kDeltaTileThreads];
    uint32_t s[kDeltaTileThreads], e[kDeltaTileThreads];
    uint32_t u0[kDeltaTileThreads], u1[kDeltaTileThreads];
    uint8_t codes[kDeltaTileThreads];
};

// One counter of endpoint w (relative rank e) in slot 0 (old, symmetric), 1 (old,
// asymmetric), 2 (new, symmetric) or 3 (new, asymmetric).
__device__ __forceinline__ void delta_bump(uint32_t *tile, int cw, uint32_t e, uint32_t slot) {
    if (cw == 0)
        atomicAdd(tile + e, 1u << (8 * slot));
    else if (cw == 1)
        atomicAdd(tile + 2 * e + (slot >> 1), 1u << (16 * (slot & 1)));
    else
        atomicAdd(tile + 4 * e + slot, 1u);
}

// Persistent blocks pop (anchor, endpoint tile) items. For its tile [lo, hi) a block
// finds, chunk by chunk, the slice of every centre row of the anchor (old centres from the
// S -> C row, inserted ones from the update list) with two binary searches, and its warps
// sweep the slices 32 entries at a time: an entry (w, c) bumps the old counter of w by the
// old codes and the new counter by the new ones (the entry's new code found among the
// updates at c, when c has any), and the insertions at c inside the tile bump new
// counters. The tile's counters then give every pair's change, counted once: at a unless
// w is touched too and ranks below a.
__global__ void __launch_bounds__(kDeltaTileThreads, 2) k_delta_tile(DeltaArgs A) {
    extern __shared__ uint4 smem_delta[];
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_delta);
    __shared__ DeltaChunk ch;
    __shared__ long long s_item;
    __shared__ long long s_red[2][kDeltaTileWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < A.tile_words; i += blockDim.x) tile[i] = 0;
    long long db = 0, du = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (long long)atomicAdd(A.next_item, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= A.n_items) break;
        // the item's anchor: the last k with toff[k] <= item
        int lo_k = 0, hi_k = A.n_anchors - 1;
        while (lo_k < hi_k) {
            const int mid = (lo_k + hi_k + 1) >> 1;
            if (A.toff[mid] <= item)
                lo_k = mid;
            else
                hi_k = mid - 1;
        }
        const int k = (int)A.order[lo_k];
        const int cw = A.cw[k];
        const uint32_t a = A.anchors[k];
        const int64_t ept = (int64_t)A.tile_words >> cw;
        const uint32_t lo = (uint32_t)((item - A.toff[lo_k]) * ept);
        const uint32_t hi = (uint32_t)((int64_t)lo + ept < A.nS ? (int64_t)lo + ept : A.nS);
        const uint32_t sb = A.seg_begin[k];
        const uint32_t se = k + 1 < A.n_anchors ? A.seg_begin[k + 1] : (uint32_t)A.n_upd;
        const int64_t rb = A.rowS_off[a], re = A.rowS_off[a + 1];
        const int64_t ncent = (re - rb) + (int64_t)(se - sb);   // old centres, then the updates
        for (int64_t cb = 0; cb < ncent; cb += kDeltaTileThreads) {
            const int64_t i = cb + tid;
            uint32_t c = 0, codes = 0, s0 = 0, s1 = 0, q0 = 0, q1 = 0;
            if (i < ncent) {
                uint32_t oa = kAbsent, na = kAbsent;
                bool use = true;
                if (i < re - rb) {
                    const uint32_t x = A.rowS[rb + i];
                    c = x & kIdMask;
                    oa = (x >> 31) ? 2u : 1u;
                    na = new_code(A, a, c, oa);
                } else {
                    const uint32_t q = sb + (uint32_t)(i - (re - rb));
                    c = A.c_by_a[q];
                    // inserted centres only (the others are old centres already)
                    use = A.old_by_a[q] == kAbsent && A.new_by_a[q] != kAbsent;
                    na = A.new_by_a[q];
                }
                if (use) {
                    const int64_t b = A.rowC_off[c], e = A.rowC_off[c + 1];
                    const int64_t p0 = lower_rank(A.rowC, b, e, lo);
                    s0 = (uint32_t)p0;
                    s1 = (uint32_t)lower_rank(A.rowC, p0, e, hi);
                    q0 = (uint32_t)lower_key(A.key, A.n_upd, (unsigned long long)c << 32);
                    q1 = (uint32_t)lower_key(A.key, A.n_upd, ((unsigned long long)c + 1) << 32);
                    codes = oa | (na << 2);
                }
            }
            ch.c[tid] = c;
            ch.s[tid] = s0;
            ch.e[tid] = s1;
            ch.u0[tid] = q0;
            ch.u1[tid] = q1;
            ch.codes[tid] = (uint8_t)codes;
            __syncthreads();
            const int nc = (int)(ncent - cb < kDeltaTileThreads ? ncent - cb : kDeltaTileThreads);
            for (int j = warp; j < nc; j += kDeltaTileWarps) {
                const uint32_t codes_j = ch.codes[j];
                if (!codes_j) continue;
                const uint32_t oa = codes_j & 3u, na = codes_j >> 2, cj = ch.c[j];
                const uint32_t u0 = ch.u0[j], u1 = ch.u1[j];
                // the old row's entries inside the tile
                for (uint32_t p = ch.s[j] + lane; p < ch.e[j]; p += 32) {
                    const uint32_t x = A.rowC[p];
                    const uint32_t w = x & kIdMask;
                    if (w == a) continue;
                    const uint32_t ow = (x >> 31) ? 2u : 1u;
                    uint32_t nw = ow;
                    if (u1 > u0) {   // an update at this centre may re-sign or delete (w, c)
                        const unsigned long long kk = ((unsigned long long)cj << 32) | w;
                        uint32_t l = u0, h = u1;
                        while (l < h) {
                            const uint32_t m = (l + h) >> 1;
                            if (A.key[m] < kk)
                                l = m + 1;
                            else
                                h = m;
                        }
                        if (l < u1 && A.key[l] == kk) nw = A.knew[l];
                    }
                    if (oa && ow) delta_bump(tile, cw, w - lo, oa == ow ? 0u : 1u);
                    if (na && nw) delta_bump(tile, cw, w - lo, na == nw ? 2u : 3u);
                }
                // insertions at this centre inside the tile
                if (na && u1 > u0) {
                    for (uint32_t q = u0 + lane; q < u1; q += 32) {
                        const uint32_t w = (uint32_t)(A.key[q] & 0xffffffffull);
                        if (w < lo || w >= hi || w == a) continue;
                        if (A.kold[q] != kAbsent || A.knew[q] == kAbsent) continue;
                        delta_bump(tile, cw, w - lo, na == A.knew[q] ? 2u : 3u);
                    }
                }
            }
            __syncthreads();
        }
        // the tile's pairs: change of f = C(p,2) + C(n,2) and of p * n; then cleared
        const uint32_t n = hi - lo;
        const uint32_t wpe = 1u << cw;
        for (uint32_t e = tid; e < n; e += kDeltaTileThreads) {
            uint32_t cnt[4];
            if (cw == 0) {
                const uint32_t v = tile[e];
                if (!v) continue;
                tile[e] = 0;
                cnt[0] = v & 0xffu;
                cnt[1] = (v >> 8) & 0xffu;
                cnt[2] = (v >> 16) & 0xffu;
                cnt[3] = v >> 24;
            } else if (cw == 1) {
                const uint32_t v0 = tile[2 * e], v1 = tile[2 * e + 1];
                if (!(v0 | v1)) continue;
                tile[2 * e] = 0;
                tile[2 * e + 1] = 0;
                cnt[0] = v0 & 0xffffu;
                cnt[1] = v0 >> 16;
                cnt[2] = v1 & 0xffffu;
                cnt[3] = v1 >> 16;
            } else {
                uint32_t *q = tile + wpe * e;
                if (!(q[0] | q[1] | q[2] | q[3])) continue;
                for (int t = 0; t < 4; ++t) {
                    cnt[t] = q[t];
                    q[t] = 0;
                }
            }
            const uint32_t w = lo + e;
            if (A.in_a[w] && w < a) continue;   // the pair is counted at w
            const long long po = cnt[0], no = cnt[1], pn = cnt[2], nn = cnt[3];
            db += (pn * (pn - 1) / 2 + nn * (nn - 1) / 2) - (po * (po - 1) / 2 + no * (no - 1) / 2);
            du += pn * nn - po * no;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        db += __shfl_xor_sync(0xffffffffu, db, o);
        du += __shfl_xor_sync(0xffffffffu, du, o);
    }
    if (lane == 0) {
        s_red[0][warp] = db;
        s_red[1][warp] = du;
    }
    __syncthreads();
    if (tid == 0) {
        long long b = 0, u = 0;
        for (int w = 0; w < kDeltaTileWarps; ++w) {
            b += s_red[0][w];
            u += s_red[1][w];
        }
        if (b) atomicAdd(A.out, (unsigned long long)b);
        if (u) atomicAdd(A.out + 1, (unsigned long long)u);
    }
}

__global__ void k_seg_end(const uint32_t *__restrict__ seg_begin, int32_t n_anchors, int64_t n_upd,
                          uint32_t *__restrict__ seg_end) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_anchors;
         k += (int64_t)gridDim.x * blockDim.x)
        seg_end[k] = k + 1 < n_anchors ? seg_begin[k + 1] : (uint32_t)n_upd;
}

__global__ void k_gather_i32(const int32_t *__restrict__ src, const uint32_t *__restrict__ order, int64_t n,
                             int32_t *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[order[i]];
}

// Device buffers released together when the owner leaves scope.
struct DeltaBuffers {
    cudaStream_t st;
    void *p[40];
    int k = 0;
    explicit DeltaBuffers(cudaStream_t s) : st(s) {}
    template <class T>
    bbc_status get(T **o, size_t cnt) {
        if (k == 40) {
            set_error("bbc_count_delta: too many scratch buffers");
            return BBC_E_INVALID_ARG;
        }
        const bbc_status s = dev_alloc_n(o, cnt, st);
        if (s == BBC_OK) p[k++] = *o;
        return s;
    }
    ~DeltaBuffers() {
        for (int i = 0; i < k; ++i) dev_free(p[i], st);
    }
};

unsigned grid_n(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

// The delta tile kernel's dynamic shared memory limit (its counter tile) on the current
// device.
bbc_status configure_delta_kernel(int tile_words) {
    static thread_local int configured = -1;
    int dev = 0;
    BBC_CUDA_TRY(cudaGetDevice(&dev));
    if (configured != dev) {
        BBC_CUDA_TRY(cudaFuncSetAttribute(k_delta_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tile_words * 4));
        configured = dev;
    }
    return BBC_OK;
}

int bits_for(int64_t n) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) < n) ++b;
    return b;
}

}  // namespace
}  // namespace bbc

using namespace bbc;

extern "C" bbc_status bbc_count_delta(const bbc_graph *g, int64_t n_updates, const int32_t *u, const int32_t *v,
                                      const int8_t *new_sign, uint32_t flags, int64_t *d_balanced,
                                      int64_t *d_unbalanced, void *cuda_stream) {
    if (!g || !d_balanced || n_updates < 0 || (n_updates > 0 && (!u || !v || !new_sign)) ||
        (flags & ~(uint32_t)BBC_INPUT_DEVICE)) {
        set_error("bbc_count_delta: NULL or inconsistent argument");
        return BBC_E_INVALID_ARG;
    }
    *d_balanced = 0;
    if (d_unbalanced) *d_unbalanced = 0;
    if (n_updates == 0) return BBC_OK;
    if (n_updates >= (int64_t)INT32_MAX) {
        set_error("bbc_count_delta: at most 2^31 - 2 updates per call");
        return BBC_E_INVALID_ARG;
    }
    try {
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        const int64_t n = n_updates, nS = g->nS, nC = g->nC;
        const int32_t n_u = g->side == 0 ? (int32_t)nS : (int32_t)nC;
        const int32_t n_v = g->side == 0 ? (int32_t)nC : (int32_t)nS;
        DeltaBuffers B(st);
        const int32_t *du = u, *dv = v;
        const int8_t *ds = new_sign;
        if (!(flags & BBC_INPUT_DEVICE)) {
            int32_t *hu = nullptr, *hv = nullptr;
            int8_t *hs = nullptr;
            BBC_TRY(B.get(&hu, (size_t)n));
            BBC_TRY(B.get(&hv, (size_t)n));
            BBC_TRY(B.get(&hs, (size_t)n));
            BBC_CUDA_TRY(cudaMemcpyAsync(hu, u, (size_t)n * 4, cudaMemcpyHostToDevice, st));
            BBC_CUDA_TRY(cudaMemcpyAsync(hv, v, (size_t)n * 4, cudaMemcpyHostToDevice, st));
            BBC_CUDA_TRY(cudaMemcpyAsync(hs, new_sign, (size_t)n, cudaMemcpyHostToDevice, st));
            du = hu;
            dv = hv;
            ds = hs;
        }
        int32_t *rankS = nullptr, *rankC = nullptr;
        uint32_t *ua = nullptr, *uc = nullptr, *k1 = nullptr, *o1 = nullptr, *k2 = nullptr, *o2 = nullptr;
        uint8_t *uold = nullptr, *unew = nullptr, *kold = nullptr, *knew = nullptr, *in_a = nullptr;
        uint8_t *old_by_a = nullptr, *new_by_a = nullptr;
        unsigned long long *key = nullptr, *out = nullptr;
        uint32_t *c_by_a = nullptr, *anchors = nullptr, *seg = nullptr;
        int32_t *first = nullptr;
        int64_t *pos = nullptr;
        unsigned *err = nullptr, *next = nullptr;
        BBC_TRY(B.get(&rankS, (size_t)std::max<int64_t>(nS, 1)));
        BBC_TRY(B.get(&rankC, (size_t)std::max<int64_t>(nC, 1)));
        BBC_TRY(B.get(&ua, (size_t)n));
        BBC_TRY(B.get(&uc, (size_t)n));
        BBC_TRY(B.get(&uold, (size_t)n));
        BBC_TRY(B.get(&unew, (size_t)n));
        BBC_TRY(B.get(&k1, (size_t)n));
        BBC_TRY(B.get(&o1, (size_t)n));
        BBC_TRY(B.get(&k2, (size_t)n));
        BBC_TRY(B.get(&o2, (size_t)n));
        BBC_TRY(B.get(&key, (size_t)n));
        BBC_TRY(B.get(&kold, (size_t)n));
        BBC_TRY(B.get(&knew, (size_t)n));
        BBC_TRY(B.get(&c_by_a, (size_t)n));
        BBC_TRY(B.get(&old_by_a, (size_t)n));
        BBC_TRY(B.get(&new_by_a, (size_t)n));
        BBC_TRY(B.get(&first, (size_t)n));
        BBC_TRY(B.get(&pos, (size_t)n + 1));
        BBC_TRY(B.get(&anchors, (size_t)n));
        BBC_TRY(B.get(&seg, (size_t)n));
        BBC_TRY(B.get(&in_a, (size_t)std::max<int64_t>(nS, 1)));
        BBC_TRY(B.get(&err, 2));
        BBC_TRY(B.get(&out, 2));
        BBC_TRY(B.get(&next, 1));
        BBC_CUDA_TRY(cudaMemsetAsync(err, 0, 8, st));
        BBC_CUDA_TRY(cudaMemsetAsync(out, 0, 16, st));
        BBC_CUDA_TRY(cudaMemsetAsync(next, 0, 4, st));
        BBC_CUDA_TRY(cudaMemsetAsync(in_a, 0, (size_t)std::max<int64_t>(nS, 1), st));
        if (nS) {
            note_launch();
            k_rank_of<<<grid_n(nS), 256, 0, st>>>(g->permS, nS, rankS);
        }
        if (nC) {
            note_launch();
            k_rank_of<<<grid_n(nC), 256, 0, st>>>(g->permC, nC, rankC);
        }
        note_launch();
        k_map_updates<<<grid_n(n), 256, 0, st>>>(du, dv, ds, n, n_u, n_v, g->side, rankS, rankC, g->rowC_off,
                                                  g->rowC, ua, uc, uold, unew, err);
        BBC_CUDA_TRY(cudaGetLastError());
        unsigned herr = 0;
        BBC_CUDA_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        if (herr & kErrRange) {
            set_error("bbc_count_delta: an update endpoint id is out of range");
            return BBC_E_OUT_OF_RANGE;
        }
        if (herr & kErrSign) {
            set_error("bbc_count_delta: a new sign other than +1, -1 or 0");
            return BBC_E_BAD_SIGN;
        }
        // a order (stable), then (c, a) order (stable sort of the a order by c)
        BBC_CUDA_TRY(cudaMemcpyAsync(k1, ua, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        note_launch();
        k_iota_u32<<<grid_n(n), 256, 0, st>>>(o1, n);
        BBC_TRY(radix_sort_pairs(k1, o1, n, bits_for(nS), st));   // k1 = a sorted, o1 = order
        note_launch();
        k_gather_u32<<<grid_n(n), 256, 0, st>>>(uc, o1, n, k2);
        BBC_CUDA_TRY(cudaMemcpyAsync(o2, o1, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        BBC_TRY(radix_sort_pairs(k2, o2, n, bits_for(nC), st));   // o2 = (c, a) order
        note_launch();
        k_check_updates<<<grid_n(n), 256, 0, st>>>(o2, ua, uc, uold, unew, n, key, kold, knew, err);
        note_launch();
        k_gather_u32<<<grid_n(n), 256, 0, st>>>(uc, o1, n, c_by_a);
        note_launch();
        k_gather_u8<<<grid_n(n), 256, 0, st>>>(uold, o1, n, old_by_a);
        note_launch();
        k_gather_u8<<<grid_n(n), 256, 0, st>>>(unew, o1, n, new_by_a);
        note_launch();
        k_anchor_marks<<<grid_n(n), 256, 0, st>>>(k1, n, first, in_a);
        BBC_TRY(exclusive_scan_i32_to_i64(first, pos, n, st));
        note_launch();
        k_anchor_list<<<grid_n(n), 256, 0, st>>>(k1, first, pos, n, anchors, seg);
        BBC_CUDA_TRY(cudaGetLastError());
        int64_t n_anchors = 0;
        BBC_CUDA_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaMemcpyAsync(&n_anchors, pos + n, 8, cudaMemcpyDeviceToHost, st));   // the total
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        if (herr & kErrDup) {
            set_error("bbc_count_delta: the same edge appears twice in one batch");
            return BBC_E_DUPLICATE_EDGE;
        }
        if (herr & kErrAbsent) {
            set_error("bbc_count_delta: a deletion of an edge the graph does not hold");
            return BBC_E_INVALID_ARG;
        }
        // work items: one per (anchor, endpoint tile), heaviest anchors first
        if (n_anchors == 0) return BBC_OK;
        const int32_t na = (int32_t)n_anchors;
        uint32_t *seg_end = nullptr, *deg_key = nullptr, *order = nullptr;
        int32_t *ntiles = nullptr, *ntiles_sorted = nullptr;
        int64_t *toff = nullptr;
        uint8_t *cw = nullptr;
        BBC_TRY(B.get(&seg_end, (size_t)na));
        BBC_TRY(B.get(&deg_key, (size_t)na));
        BBC_TRY(B.get(&order, (size_t)na));
        BBC_TRY(B.get(&ntiles, (size_t)na));
        BBC_TRY(B.get(&ntiles_sorted, (size_t)na));
        BBC_TRY(B.get(&toff, (size_t)na + 1));
        BBC_TRY(B.get(&cw, (size_t)na));
        const Tuning T = resolve_tuning(nullptr, device_sm_count());
        DeltaArgs A{g->rowS_off, g->rowS, g->rowC_off, g->rowC, nS, key, kold, knew, n,
                    c_by_a, old_by_a, new_by_a, anchors, seg, na, in_a,
                    order, toff, cw, 0, T.tile_words, next, out};
        note_launch();
        k_seg_end<<<grid_n(na), 256, 0, st>>>(seg, na, n, seg_end);
        note_launch();
        k_delta_plan<<<grid_n(na), 256, 0, st>>>(A, seg_end, ntiles, cw, deg_key);
        note_launch();
        k_iota_u32<<<grid_n(na), 256, 0, st>>>(order, na);
        BBC_TRY(radix_sort_pairs(deg_key, order, na, 32, st));
        note_launch();
        k_gather_i32<<<grid_n(na), 256, 0, st>>>(ntiles, order, na, ntiles_sorted);
        BBC_TRY(exclusive_scan_i32_to_i64(ntiles_sorted, toff, na, st));
        int64_t n_items = 0;
        BBC_CUDA_TRY(cudaMemcpyAsync(&n_items, toff + na, 8, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        A.n_items = n_items;
        BBC_TRY(configure_delta_kernel(T.tile_words));
        const int blocks = (int)std::min<int64_t>(n_items, (int64_t)device_sm_count() * 2);
        note_launch();
        k_delta_tile<<<blocks, kDeltaTileThreads, (size_t)T.tile_words * 4, st>>>(A);
        BBC_CUDA_TRY(cudaGetLastError());
        unsigned long long h[2] = {0, 0};
        BBC_CUDA_TRY(cudaMemcpyAsync(h, out, 16, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        *d_balanced = (int64_t)h[0];
        if (d_unbalanced) *d_unbalanced = (int64_t)h[1];
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_count_delta");
        return BBC_E_CUDA;
    }
}
