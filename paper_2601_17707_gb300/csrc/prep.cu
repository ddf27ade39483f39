// prep.cu -- graph preparation on the device (bbc_prepare).
//
// Steps, all in this file's kernels plus the radix sort / scan of sort_scan.cu:
//   1. validate ids and signs, count degrees (k_validate_degrees);
//   2. per side sum of C(d, 2) and max degree (k_degree_stats) -> the pair side S is
//      the side whose opposite side has the smaller sum (that sum is W, the number of
//      oriented wedges the count visits);
//   3. rank S and C by (degree descending, id descending), the vertex priority of
//      Def. 6 (k_rank_keys + stable radix sort + k_invert_perm);
//   4. map every edge to (rank_S, rank_C | sign << 31) and sort it twice, stably:
//      by rank_S (giving the S -> C rows) and then by rank_C (giving the C -> S rows,
//      each sorted by anchor rank because the input of the second sort is already in
//      rank_S order); duplicates are adjacent there (k_count_duplicates);
//   5. row offsets by exclusive scans of the ranked degrees;
//   6. per anchor the number of oriented wedges it visits (k_wedge_estimate), then the
//      work lists (k_classify + k_emit_items + a cost-ordered radix sort), heavy first
//      as in the fanout ordering of Algorithm 4.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "graph.cuh"

namespace bbc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int threads = kThreads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 32;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

inline int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

__global__ void k_validate_degrees(const int32_t *__restrict__ u, const int32_t *__restrict__ v,
                                   const int8_t *__restrict__ s, int64_t n, int32_t n_u,
                                   int32_t n_v, int32_t *__restrict__ deg_u,
                                   int32_t *__restrict__ deg_v, unsigned *__restrict__ err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = u[i], b = v[i];
        const int8_t sg = s[i];
        unsigned bad = 0;
        if (a < 0 || a >= n_u || b < 0 || b >= n_v) bad |= 1u;
        if (sg != 1 && sg != -1) bad |= 2u;
        if (bad) {
            atomicOr(err, bad);
            continue;
        }
        // lanes of one warp that hit the same vertex add once (edge lists sorted by one
        // side put a hub's edges in consecutive lanes)
        const unsigned act = __activemask();
        const int lane = threadIdx.x & 31;
        const unsigned mu = __match_any_sync(act, a);
        if (lane == __ffs(mu) - 1) atomicAdd(deg_u + a, __popc(mu));
        const unsigned mv = __match_any_sync(act, b);
        if (lane == __ffs(mv) - 1) atomicAdd(deg_v + b, __popc(mv));
    }
}

// stats[0] += sum C(d, 2) (uint64), stats[1] = max d (as uint64 via atomicMax)
__global__ void k_degree_stats(const int32_t *__restrict__ deg, int64_t n,
                               unsigned long long *__restrict__ stats) {
    unsigned long long s = 0, m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long d = (unsigned long long)deg[i];
        s += d * (d - (d > 0)) / 2;
        m = d > m ? d : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(kFull, s, o);
        const unsigned long long mo = __shfl_down_sync(kFull, m, o);
        m = mo > m ? mo : m;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(stats + 0, s);
        atomicMax(stats + 1, m);
    }
}

// keys[i] = maxdeg - deg[id], vals[i] = id, with id = n - 1 - i: a stable ascending sort
// then lists ids by degree descending and, among equal degrees, id descending.
__global__ void k_rank_keys(const int32_t *__restrict__ deg, int64_t n, int32_t maxdeg,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t id = n - 1 - i;
        keys[i] = (uint32_t)(maxdeg - deg[id]);
        vals[i] = (uint32_t)id;
    }
}

__global__ void k_invert_perm(const uint32_t *__restrict__ perm, int64_t n,
                              int32_t *__restrict__ rank, int32_t *__restrict__ perm_out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t id = perm[r];
        rank[id] = (int32_t)r;
        perm_out[r] = (int32_t)id;
    }
}

__global__ void k_gather_deg(const int32_t *__restrict__ deg, const int32_t *__restrict__ perm,
                             int64_t n, int32_t *__restrict__ out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        out[r] = deg[perm[r]];
}

__global__ void k_map_edges(const int32_t *__restrict__ u, const int32_t *__restrict__ v,
                            const int8_t *__restrict__ s, int64_t n, int side,
                            const int32_t *__restrict__ rankS, const int32_t *__restrict__ rankC,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t sid = side == 0 ? u[i] : v[i];
        const int32_t cid = side == 0 ? v[i] : u[i];
        keys[i] = (uint32_t)rankS[sid];
        vals[i] = (uint32_t)rankC[cid] | (s[i] < 0 ? kSignBit : 0u);
    }
}

// (rank_S, rank_C | sign) -> (rank_C, rank_S | sign)
__global__ void k_swap_sides(const uint32_t *__restrict__ ka, const uint32_t *__restrict__ va,
                             int64_t n, uint32_t *__restrict__ kb, uint32_t *__restrict__ vb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = va[i];
        kb[i] = x & kIdMask;
        vb[i] = ka[i] | (x & kSignBit);
    }
}

__global__ void k_count_duplicates(const uint32_t *__restrict__ kc, const uint32_t *__restrict__ vc,
                                   int64_t n, unsigned long long *__restrict__ dups) {
    unsigned long long c = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (kc[j] == kc[j - 1] && ((vc[j] ^ vc[j - 1]) & kIdMask) == 0) ++c;
    }
    if (c) atomicAdd(dups, c);
}

// Keeps the last entry of every run of equal (rank_C, rank_S) -- the last occurrence in
// input order, since both sorts are stable -- and writes it back as an original-id edge.
__global__ void k_dedup_last(const uint32_t *__restrict__ kc, const uint32_t *__restrict__ vc,
                             int64_t n, const int64_t *__restrict__ pos, int side,
                             const int32_t *__restrict__ permS, const int32_t *__restrict__ permC,
                             int32_t *__restrict__ u, int32_t *__restrict__ v,
                             int8_t *__restrict__ s) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const bool last = j == n - 1 || kc[j + 1] != kc[j] || ((vc[j + 1] ^ vc[j]) & kIdMask) != 0;
        if (!last) continue;
        const int64_t o = pos[j];
        const int32_t cid = permC[kc[j]];
        const int32_t sid = permS[vc[j] & kIdMask];
        u[o] = side == 0 ? sid : cid;
        v[o] = side == 0 ? cid : sid;
        s[o] = (vc[j] & kSignBit) ? (int8_t)-1 : (int8_t)1;
    }
}

__global__ void k_last_flags(const uint32_t *__restrict__ kc, const uint32_t *__restrict__ vc,
                             int64_t n, int32_t *__restrict__ flag) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        flag[j] = (j == n - 1 || kc[j + 1] != kc[j] || ((vc[j + 1] ^ vc[j]) & kIdMask) != 0) ? 1 : 0;
}

__device__ __forceinline__ int64_t lower_bound_rank(const uint32_t *__restrict__ row, int64_t b,
                                                    int64_t e, uint32_t key) {
    while (b < e) {
        const int64_t m = (b + e) >> 1;
        if ((__ldg(row + m) & kIdMask) < key)
            b = m + 1;
        else
            e = m;
    }
    return b;
}

// wl[a] = number of oriented wedges at anchor a: for every entry (a, c) of the S -> C
// rows, the entries of row c of higher (orient_low: lower) rank than a. The rows are
// grouped by anchor, so a segmented warp sum leaves one atomic per anchor run. The
// anchor's endpoint range inside row c (the entries after a, or before a with orient_low)
// is kept as rng[e], so the counting kernels find every slice without a row-offset load.
__global__ void k_wedge_estimate(const uint32_t *__restrict__ anchor_of, const uint32_t *__restrict__ rowS,
                                 int64_t n, const int64_t *__restrict__ rowC_off,
                                 const uint32_t *__restrict__ rowC, int orient_low,
                                 unsigned long long *__restrict__ wl, uint2 *__restrict__ rng) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t e = base + threadIdx.x;
        const bool valid = e < n;
        uint32_t a = 0xffffffffu;
        unsigned long long cnt = 0;
        if (valid) {
            a = anchor_of[e];
            const uint32_t c = rowS[e] & kIdMask;
            const int64_t b = rowC_off[c], en = rowC_off[c + 1];
            const int64_t p = lower_bound_rank(rowC, b, en, a);
            rng[e] = orient_low ? make_uint2((uint32_t)b, (uint32_t)p)
                                : make_uint2((uint32_t)p + 1u, (uint32_t)en);
            cnt = orient_low ? (unsigned long long)(p - b) : (unsigned long long)(en - p - 1);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, cnt, o);
            const uint32_t ka = __shfl_up_sync(kFull, a, o);
            if (lane >= o && ka == a) cnt += y;
        }
        const uint32_t next = __shfl_down_sync(kFull, a, 1);
        if (valid && (lane == 31 || next != a) && cnt) atomicAdd(wl + a, cnt);
    }
}

struct ClassifyParams {
    int32_t nS;
    int orient_low;
    int tile_words;
    int warp_max;
    long long split;
    int warp_tiles;            // single-tile anchors that fit a warp's table go to k_warp_tile
    int var_width;             // block tiles choose their counter width tile by tile
    int group_warps;           // warps per group-tile table (its capacity)
    int centre_split;          // anchors heavier than their tiles can spread are split by centres too
};

// A centre-split tile is cut into parts of about split / kCentreSplitDiv wedges: finer than
// the tile split, since these anchors are the ones that would otherwise end the launch
// alone. Each part keeps at least kMinPartCentres centres.
constexpr long long kCentreSplitDiv = 16;
constexpr long long kMinPartCentres = 1024;

// Work of one anchor: kind 0 none, 1 warp-hash item, 2 tile items, 3 warp-tile item (its
// whole endpoint range fits one warp's counter table), 4 group-tile item (it fits a group
// of warps' pooled table). For tiles: the counter width code (largest reachable count
// min(degree, wedges) <= 255 / 65535 / more, or kWidthPerTile when the widths are chosen
// tile by tile), the number of tiles over its endpoint range (not counted, and left at 1,
// when count_tiles is false), how many tile ranges they are split into, and into how many
// centre parts each tile is cut (1, or >= 2 for a centre-split anchor: then every tile is
// its own range and the anchor has groups * parts items).
__device__ __forceinline__ void classify_one(const ClassifyParams &P, const int64_t *__restrict__ rowS_off,
                                             unsigned long long wl, int64_t deg, int a, int *kind, int *cw,
                                             int *ntiles, int *groups, int *parts, bool count_tiles = true) {
    *kind = 0;
    *cw = 0;
    *ntiles = 0;
    *groups = 0;
    *parts = 1;
    if (wl == 0 || deg < 2) return;
    if ((long long)wl <= P.warp_max) {
        *kind = 1;
        return;
    }
    const long long maxcount = deg < (long long)wl ? deg : (long long)wl;
    const int w = width_for_bound((unsigned long long)maxcount);
    const long long span = P.orient_low ? a : (long long)P.nS - 1 - a;
    // with 8-bit counters a table starts at an even endpoint, one slot early for an odd
    // first endpoint, so it holds two endpoints less than its size to be safe
    const long long slack = w == 0 ? 2 : 0;
    if (P.warp_tiles && span + slack <= (long long)group_tile_endpoints(1, w)) {
        *kind = 3;
        *cw = w;
        *ntiles = 1;
        *groups = 1;
        return;
    }
    if (P.warp_tiles && span + slack <= (long long)group_tile_endpoints(P.group_warps, w)) {
        *kind = 4;
        *cw = w;
        *ntiles = 1;
        *groups = 1;
        return;
    }
    int nt;
    if (P.var_width) {
        const uint32_t range_lo = P.orient_low ? 0u : (uint32_t)a + 1u;
        const uint32_t range_hi = P.orient_low ? (uint32_t)a : (uint32_t)P.nS;
        nt = count_tiles ? var_tile_count(rowS_off, (unsigned long long)maxcount, range_lo, range_hi,
                                          (uint32_t)P.tile_words)
                         : 1;
        *cw = kWidthPerTile;
    } else {
        const long long ept = tile_endpoints(w, (uint32_t)P.tile_words);
        nt = (int)((span + ept - 1) / ept);
        *cw = w;
    }
    long long g = 1;
    if ((long long)wl > P.split) g = ((long long)wl + P.split - 1) / P.split;
    if (P.centre_split && count_tiles && 2 * g > nt) {
        // the tile ranges it wants (ceil(wl / split)) are more than half its tiles: cut
        // every tile's centres too, into parts of about split / kCentreSplitDiv wedges
        // (an anchor too light for two parts stays whole)
        const long long per_part = P.split / kCentreSplitDiv > 0 ? P.split / kCentreSplitDiv : 1;
        long long k = ((long long)wl + (long long)nt * per_part - 1) / ((long long)nt * per_part);
        if (k > kMaxParts) k = kMaxParts;
        if (k > deg / kMinPartCentres) k = deg / kMinPartCentres;
        if (k >= 2) *parts = (int)k;
    }
    if (g > nt) g = nt;
    *kind = 2;
    *ntiles = nt;
    *groups = (int)g;
}

__global__ void k_classify(ClassifyParams P, const unsigned long long *__restrict__ wl,
                           const int64_t *__restrict__ rowS_off, int32_t *__restrict__ n_tile,
                           int32_t *__restrict__ n_warp, int64_t *__restrict__ n_bnd,
                           int32_t *__restrict__ n_wt, int32_t *__restrict__ n_gt,
                           int32_t *__restrict__ n_csg) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < P.nS;
         a += (int64_t)gridDim.x * blockDim.x) {
        int kind, cw, nt, g, k;
        const int64_t deg = rowS_off[a + 1] - rowS_off[a];
        classify_one(P, rowS_off, wl[a], deg, (int)a, &kind, &cw, &nt, &g, &k);
        n_tile[a] = kind == 2 ? (k > 1 ? nt * k : g) : 0;
        n_csg[a] = kind == 2 && k > 1 ? nt : 0;
        n_warp[a] = kind == 1 ? 1 : 0;
        n_wt[a] = kind == 3 ? 1 : 0;
        n_gt[a] = kind == 4 ? 1 : 0;
        n_bnd[a] = kind == 2 && nt > 1 ? deg * (nt - 1) : 0;
    }
}

// Interior tile boundaries: for every S -> C entry (a, c) of a tile anchor, the index in
// row c of the first endpoint of each of a's tiles 1 .. tiles-1 (the same tile walk as the
// tile kernel's, with per-tile widths when the item says so), found by galloping from
// the previous boundary. One thread per entry; the layout (boundary-major per anchor)
// lets the tile kernel read them coalesced.
__global__ void k_tile_bounds(ClassifyParams P, const unsigned long long *__restrict__ wl,
                              const int64_t *__restrict__ rowS_off,
                              const uint32_t *__restrict__ anchor_of, const uint2 *__restrict__ rng,
                              const uint32_t *__restrict__ rowC, const int64_t *__restrict__ boff,
                              int64_t n, uint32_t *__restrict__ bnd) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = anchor_of[e];
        const int64_t sb = rowS_off[a], deg = rowS_off[a + 1] - sb;
        int kind, cw, nt, g, k;
        classify_one(P, rowS_off, wl[a], deg, (int)a, &kind, &cw, &nt, &g, &k, false);
        if (kind != 2) continue;
        const uint32_t range_lo = P.orient_low ? 0u : a + 1u;
        const uint32_t range_hi = P.orient_low ? a : (uint32_t)P.nS;
        const unsigned long long bound = deg < (long long)wl[a] ? (unsigned long long)deg : wl[a];
        const uint32_t ept = tile_endpoints(cw == kWidthPerTile ? 0 : cw, (uint32_t)P.tile_words);
        if (cw != kWidthPerTile) nt = (int)((range_hi - range_lo + ept - 1) / ept);
        uint32_t next = cw == kWidthPerTile
                            ? var_tile_at(rowS_off, bound, range_lo, range_hi, (uint32_t)P.tile_words).hi
                            : range_lo + ept;
        if (next >= range_hi) continue;   // a single tile: no interior boundary
        const uint2 r = rng[e];
        uint32_t pos = r.x;
        uint32_t *dst = bnd + boff[a] + (e - sb);
        for (int t = 1; next < range_hi; ++t) {
            const uint32_t key = next;
            next = cw == kWidthPerTile ? var_tile_at(rowS_off, bound, key, range_hi, (uint32_t)P.tile_words).hi
                                       : key + ept;
            uint32_t lo = pos, step = 1;
            while (lo + step <= r.y && (__ldg(rowC + lo + step - 1) & kIdMask) < key) {
                lo += step;
                step <<= 1;
            }
            uint32_t hi = min(lo + step - 1, r.y);
            while (lo < hi) {
                const uint32_t m = (lo + hi) >> 1;
                if ((__ldg(rowC + m) & kIdMask) < key)
                    lo = m + 1;
                else
                    hi = m;
            }
            pos = lo;
            dst[(int64_t)(t - 1) * deg] = pos;
        }
    }
}

// Writes the items and, per tile item, a 16-bit sort key that orders items by their
// expected wedge count, largest first (the fanout ordering of Algorithm 4).
__global__ void k_emit_items(ClassifyParams P, const unsigned long long *__restrict__ wl,
                             const int64_t *__restrict__ rowS_off, const int64_t *__restrict__ pos_tile,
                             const int64_t *__restrict__ pos_warp, const int64_t *__restrict__ pos_wt,
                             const int64_t *__restrict__ pos_gt, const int64_t *__restrict__ pos_csg,
                             const int64_t *__restrict__ pos_csi, TileItem *__restrict__ tiles,
                             uint32_t *__restrict__ keys, HashItem *__restrict__ warp,
                             HashItem *__restrict__ wt, HashItem *__restrict__ gt,
                             CentreSplit *__restrict__ cs_desc, TileItem *__restrict__ cs_items) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < P.nS;
         a += (int64_t)gridDim.x * blockDim.x) {
        int kind, cw, nt, g, k;
        const unsigned long long w = wl[a];
        classify_one(P, rowS_off, w, rowS_off[a + 1] - rowS_off[a], (int)a, &kind, &cw, &nt, &g, &k);
        if (kind == 1) {
            warp[pos_warp[a]] = HashItem{0, (int32_t)a, (int32_t)w, 0};
        } else if (kind == 3 || kind == 4) {
            const HashItem h{0, (int32_t)a, (int32_t)(w > 0x7fffffffull ? 0x7fffffff : w), cw};
            if (kind == 3)
                wt[pos_wt[a]] = h;
            else
                gt[pos_gt[a]] = h;
        } else if (kind == 2 && k > 1) {
            // centre-split: item (tile t, part p) at t * k + p, in both lists; its record
            // sits at the same index of the centre-split list
            TileItem *dst = tiles + pos_tile[a];
            uint32_t *kd = keys + pos_tile[a];
            const double cost = (double)w / ((double)nt * k) + 1.0;
            int q = (int)(log2(cost) * 1024.0);
            q = q < 0 ? 0 : (q > 65535 ? 65535 : q);
            for (int t = 0; t < nt; ++t) {
                for (int p = 0; p < k; ++p) {
                    const int64_t ci = pos_csi[a] + (int64_t)t * k + p;
                    cs_desc[ci] = CentreSplit{t, (int16_t)p, (int16_t)k, (int32_t)(pos_csg[a] + t), 0};
                    const TileItem it{0, (int32_t)a, (int32_t)ci, pack_tile_end(t + 1, cw) | kCentreSplitBit};
                    dst[t * k + p] = it;
                    kd[t * k + p] = 65535u - (uint32_t)q;
                    cs_items[ci] = it;
                }
            }
        } else if (kind == 2) {
            TileItem *dst = tiles + pos_tile[a];
            uint32_t *kd = keys + pos_tile[a];
            for (int i = 0; i < g; ++i) {
                const int t0 = (int)((long long)nt * i / g);
                const int t1 = (int)((long long)nt * (i + 1) / g);
                dst[i] = TileItem{0, (int32_t)a, t0, pack_tile_end(t1, cw)};
                const double cost = (double)w * (double)(t1 - t0) / (double)nt + 1.0;
                int q = (int)(log2(cost) * 1024.0);
                q = q < 0 ? 0 : (q > 65535 ? 65535 : q);
                kd[i] = 65535u - (uint32_t)q;
            }
        }
    }
}

// Items on the centre-split list per anchor: all of a centre-split anchor's tile items.
__global__ void k_cs_items(const int32_t *__restrict__ n_tile, const int32_t *__restrict__ n_csg,
                           int32_t *__restrict__ n_csi, int64_t n) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x)
        n_csi[a] = n_csg[a] > 0 ? n_tile[a] : 0;
}

__global__ void k_iota(uint32_t *__restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (uint32_t)i;
}

__global__ void k_gather_items(const TileItem *__restrict__ in, const uint32_t *__restrict__ order,
                               int64_t n, TileItem *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[order[i]];
}

// --------------------------------------------------------------------------- host helpers

// Frees a list of pool allocations at scope exit.
struct Scratch {
    cudaStream_t st;
    void *p[32];
    int n = 0;
    explicit Scratch(cudaStream_t s) : st(s) {}
    template <class T>
    bbc_status get(T **out, size_t count) {
        bbc_status s = dev_alloc_n(out, count, st);
        if (s == BBC_OK) p[n++] = *out;
        return s;
    }
    ~Scratch() {
        for (int i = 0; i < n; ++i) dev_free(p[i], st);
    }
};

#define BBC_LAUNCH_CHECK(what)                                       \
    do {                                                             \
        cudaError_t _e = cudaGetLastError();                         \
        if (_e != cudaSuccess) return ::bbc::cuda_fail(_e, what);    \
    } while (0)

// Ranks the vertices of one side by Def. 6; writes rank[id] and perm[rank] = id.
bbc_status rank_side(const int32_t *deg, int64_t n, int32_t maxdeg, int32_t *rank, int32_t *perm,
                     cudaStream_t st) {
    if (n == 0) return BBC_OK;
    Scratch sc(st);
    uint32_t *k = nullptr, *vv = nullptr;
    BBC_TRY(sc.get(&k, (size_t)n));
    BBC_TRY(sc.get(&vv, (size_t)n));
    note_launch();
    k_rank_keys<<<grid_for(n), kThreads, 0, st>>>(deg, n, maxdeg, k, vv);
    BBC_LAUNCH_CHECK("k_rank_keys");
    BBC_TRY(radix_sort_pairs(k, vv, n, bit_length((uint64_t)maxdeg), st));
    note_launch();
    k_invert_perm<<<grid_for(n), kThreads, 0, st>>>(vv, n, rank, perm);
    BBC_LAUNCH_CHECK("k_invert_perm");
    return BBC_OK;
}

}  // namespace

DevGraph host_descriptor(const bbc_graph *g, bool per_vertex, bool with_bounds) {
    DevGraph d{};
    d.rowS_off = g->rowS_off;
    d.rowS = g->rowS;
    d.rowC_off = g->rowC_off;
    d.rowC = g->rowC;
    d.nS = g->nS;
    d.nC = g->nC;
    d.orient_low = g->orient_low;
    d.bS = per_vertex ? g->bS : nullptr;
    d.bC = per_vertex ? g->bC : nullptr;
    d.totals = g->totals;
    d.wl = g->wl;
    d.rng = g->rng;
    d.bnd = with_bounds ? g->bnd : nullptr;
    d.boff = with_bounds ? g->boff : nullptr;
    d.cs_desc = g->cs_desc;
    d.cs_buf = g->cs_buf;
    d.cs_arrive = g->cs_arrive;
    d.cs_group_words = g->cs_group_words;
    return d;
}

bbc_status clear_centre_split(const bbc_graph *g, cudaStream_t st) {
    if (g->n_cs_groups == 0) return BBC_OK;
    BBC_CUDA_TRY(cudaMemsetAsync(g->cs_buf, 0, (size_t)(g->n_cs_groups * g->cs_group_words) * 4, st));
    BBC_CUDA_TRY(cudaMemsetAsync(g->cs_arrive, 0, (size_t)g->n_cs_groups * 4, st));
    return BBC_OK;
}

void release_graph(bbc_graph *g, cudaStream_t st) {
    if (!g) return;
    void *ptrs[] = {g->rowS_off, g->rowS, g->rowC_off, g->rowC, g->permS, g->permC, g->wl, g->rng, g->anchor_of, g->bnd, g->boff,
                    g->tile_items, g->warp_items, g->wt_items, g->gt_items, g->dgraph, g->bS, g->bC,
                    g->totals, g->queue, g->cs_desc, g->cs_items, g->cs_buf, g->cs_arrive};
    for (void *p : ptrs)
        if (p) dev_free(p, st);
    delete g;
}

bbc_status build_work_lists(bbc_graph *g, const Tuning &t, cudaStream_t st) {
    if (g->items_valid && g->items_tuning.tile_words == t.tile_words &&
        g->items_tuning.warp_max_wedges == t.warp_max_wedges &&
        g->items_tuning.split_wedges == t.split_wedges && g->items_tuning.plain == t.plain &&
        g->items_tuning.tiles_only == t.tiles_only && g->items_tuning.group_warps == t.group_warps)
        return BBC_OK;
    if (g->tile_items) dev_free(g->tile_items, st);
    if (g->warp_items) dev_free(g->warp_items, st);
    if (g->wt_items) dev_free(g->wt_items, st);
    g->wt_items = nullptr;
    g->n_wt = 0;
    if (g->gt_items) dev_free(g->gt_items, st);
    g->gt_items = nullptr;
    g->n_gt = 0;
    if (g->bnd) dev_free(g->bnd, st);
    if (g->boff) dev_free(g->boff, st);
    if (g->cs_desc) dev_free(g->cs_desc, st);
    if (g->cs_items) dev_free(g->cs_items, st);
    if (g->cs_buf) dev_free(g->cs_buf, st);
    if (g->cs_arrive) dev_free(g->cs_arrive, st);
    g->cs_desc = nullptr;
    g->cs_items = nullptr;
    g->cs_buf = nullptr;
    g->cs_arrive = nullptr;
    g->n_cs_items = 0;
    g->n_cs_groups = 0;
    g->tile_items = nullptr;
    g->warp_items = nullptr;
    g->bnd = nullptr;
    g->boff = nullptr;
    g->n_tile = g->n_warp = 0;
    g->items_valid = false;
    g->layout_version++;
    const int64_t nS = g->nS;
    if (nS == 0) {
        g->items_tuning = t;
        g->items_valid = true;
        return BBC_OK;
    }
    Scratch sc(st);
    int32_t *nt = nullptr, *nh = nullptr, *nw = nullptr, *ng = nullptr, *ncg = nullptr;
    int64_t *pt = nullptr, *ph = nullptr, *pw = nullptr, *pg = nullptr, *nb = nullptr, *pcg = nullptr,
            *pci = nullptr;
    BBC_TRY(sc.get(&ncg, (size_t)nS));
    BBC_TRY(sc.get(&pcg, (size_t)nS + 1));
    BBC_TRY(sc.get(&pci, (size_t)nS + 1));
    BBC_TRY(sc.get(&nt, (size_t)nS));
    BBC_TRY(sc.get(&nh, (size_t)nS));
    BBC_TRY(sc.get(&nw, (size_t)nS));
    BBC_TRY(sc.get(&ng, (size_t)nS));
    BBC_TRY(sc.get(&pt, (size_t)nS + 1));
    BBC_TRY(sc.get(&ph, (size_t)nS + 1));
    BBC_TRY(sc.get(&pw, (size_t)nS + 1));
    BBC_TRY(sc.get(&pg, (size_t)nS + 1));
    BBC_TRY(sc.get(&nb, (size_t)nS));
    BBC_TRY(dev_alloc_n(&g->boff, (size_t)nS + 1, st));
    ClassifyParams P{g->nS, g->orient_low, t.tile_words, t.warp_max_wedges, t.split_wedges,
                     (t.plain || t.tiles_only) ? 0 : 1, t.tiles_only ? 0 : 1, t.group_warps,
                     (t.plain || t.tiles_only) ? 0 : 1};
    // one tile group's merged counters: two per endpoint of the widest tile
    const int64_t group_words = 2 * (int64_t)tile_endpoints(0, (uint32_t)t.tile_words);
    int64_t n_csg = 0;
    for (;;) {
        note_launch();
        k_classify<<<grid_for(nS), kThreads, 0, st>>>(P, g->wl, g->rowS_off, nt, nh, nb, nw, ng, ncg);
        BBC_LAUNCH_CHECK("k_classify");
        if (!P.centre_split) break;
        BBC_TRY(exclusive_scan_i32_to_i64(ncg, pcg, nS, st));
        BBC_CUDA_TRY(cudaMemcpyAsync(&n_csg, pcg + nS, 8, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        // the merge buffers stay below 8 bytes per edge (and 16 MiB for small graphs);
        // past that the anchors keep their tile split only
        const int64_t cap = std::max<int64_t>(int64_t(16) << 20, 8 * g->n_edges);
        if (n_csg * group_words * 4 <= cap) break;
        P.centre_split = 0;
        n_csg = 0;
    }
    int64_t n_csi = 0;
    if (n_csg > 0) {
        // a centre-split anchor's items (all of its n_tile) also form the centre-split list
        int32_t *nci = nullptr;
        BBC_TRY(sc.get(&nci, (size_t)nS));
        note_launch();
        k_cs_items<<<grid_for(nS), kThreads, 0, st>>>(nt, ncg, nci, nS);
        BBC_LAUNCH_CHECK("k_cs_items");
        BBC_TRY(exclusive_scan_i32_to_i64(nci, pci, nS, st));
        BBC_CUDA_TRY(cudaMemcpyAsync(&n_csi, pci + nS, 8, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        if (n_csi > INT32_MAX) {
            set_error("work list longer than 2^31 items");
            return BBC_E_INVALID_ARG;
        }
        BBC_TRY(dev_alloc_n(&g->cs_desc, (size_t)n_csi, st));
        BBC_TRY(dev_alloc_n(&g->cs_items, (size_t)n_csi, st));
        BBC_TRY(dev_alloc_n(&g->cs_buf, (size_t)(n_csg * group_words), st));
        BBC_TRY(dev_alloc_n(&g->cs_arrive, (size_t)n_csg, st));
        g->n_cs_items = (int32_t)n_csi;
        g->n_cs_groups = n_csg;
        g->cs_group_words = group_words;
    }
    BBC_TRY(exclusive_scan_i32_to_i64(nt, pt, nS, st));
    BBC_TRY(exclusive_scan_i32_to_i64(nh, ph, nS, st));
    BBC_TRY(exclusive_scan_i32_to_i64(nw, pw, nS, st));
    BBC_TRY(exclusive_scan_i32_to_i64(ng, pg, nS, st));
    BBC_TRY(exclusive_scan_i64(nb, g->boff, nS, st));
    int64_t counts[5];
    BBC_CUDA_TRY(cudaMemcpyAsync(&counts[0], pt + nS, 8, cudaMemcpyDeviceToHost, st));
    BBC_CUDA_TRY(cudaMemcpyAsync(&counts[1], ph + nS, 8, cudaMemcpyDeviceToHost, st));
    BBC_CUDA_TRY(cudaMemcpyAsync(&counts[2], g->boff + nS, 8, cudaMemcpyDeviceToHost, st));
    BBC_CUDA_TRY(cudaMemcpyAsync(&counts[3], pw + nS, 8, cudaMemcpyDeviceToHost, st));
    BBC_CUDA_TRY(cudaMemcpyAsync(&counts[4], pg + nS, 8, cudaMemcpyDeviceToHost, st));
    BBC_CUDA_TRY(cudaStreamSynchronize(st));
    if (counts[3] > INT32_MAX || counts[4] > INT32_MAX) {
        set_error("work list longer than 2^31 items");
        return BBC_E_INVALID_ARG;
    }
    BBC_TRY(dev_alloc_n(&g->wt_items, (size_t)counts[3], st));
    g->n_wt = (int32_t)counts[3];
    BBC_TRY(dev_alloc_n(&g->gt_items, (size_t)counts[4], st));
    g->n_gt = (int32_t)counts[4];
    BBC_TRY(dev_alloc_n(&g->bnd, (size_t)counts[2], st));
    if (counts[2] > 0 && g->n_edges > 0) {
        note_launch();
        k_tile_bounds<<<grid_for(g->n_edges), kThreads, 0, st>>>(
            P, g->wl, g->rowS_off, g->anchor_of, g->rng, g->rowC, g->boff, g->n_edges, g->bnd);
        BBC_LAUNCH_CHECK("k_tile_bounds");
    }
    if (counts[0] > INT32_MAX || counts[1] > INT32_MAX) {
        set_error("work list longer than 2^31 items");
        return BBC_E_INVALID_ARG;
    }
    const int64_t ntile = counts[0];
    TileItem *raw = nullptr;
    uint32_t *keys = nullptr;
    BBC_TRY(sc.get(&raw, (size_t)ntile));
    BBC_TRY(sc.get(&keys, (size_t)ntile));
    BBC_TRY(dev_alloc_n(&g->warp_items, (size_t)counts[1], st));
    g->n_warp = (int32_t)counts[1];
    BBC_TRY(dev_alloc_n(&g->tile_items, (size_t)ntile, st));
    g->n_tile = (int32_t)ntile;
    note_launch();
    k_emit_items<<<grid_for(nS), kThreads, 0, st>>>(P, g->wl, g->rowS_off, pt, ph, pw, pg, pcg, pci, raw, keys,
                                                     g->warp_items, g->wt_items, g->gt_items, g->cs_desc,
                                                     g->cs_items);
    BBC_LAUNCH_CHECK("k_emit_items");
    // Order the tile items by expected cost, largest first (the plain schedule keeps
    // rank order).
    if (ntile > 0 && t.plain) {
        BBC_CUDA_TRY(cudaMemcpyAsync(g->tile_items, raw, sizeof(TileItem) * (size_t)ntile,
                                     cudaMemcpyDeviceToDevice, st));
    } else if (ntile > 0) {
        uint32_t *order = nullptr;
        BBC_TRY(sc.get(&order, (size_t)ntile));
        note_launch();
        k_iota<<<grid_for(ntile), kThreads, 0, st>>>(order, ntile);
        BBC_LAUNCH_CHECK("k_iota");
        BBC_TRY(radix_sort_pairs(keys, order, ntile, 16, st));
        note_launch();
        k_gather_items<<<grid_for(ntile), kThreads, 0, st>>>(raw, order, ntile, g->tile_items);
        BBC_LAUNCH_CHECK("k_gather_items");
    }
    g->items_tuning = t;
    g->items_valid = true;
    return BBC_OK;
}

bbc_status prepare_graph(int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *u,
                         const int32_t *v, const int8_t *sign, uint32_t flags, cudaStream_t st,
                         bbc_graph **out) {
    Scratch sc(st);
    const int32_t *du = u, *dv = v;
    const int8_t *ds = sign;
    if (!(flags & BBC_INPUT_DEVICE) && n_edges > 0) {
        int32_t *hu = nullptr, *hv = nullptr;
        int8_t *hs = nullptr;
        BBC_TRY(sc.get(&hu, (size_t)n_edges));
        BBC_TRY(sc.get(&hv, (size_t)n_edges));
        BBC_TRY(sc.get(&hs, (size_t)n_edges));
        BBC_CUDA_TRY(cudaMemcpyAsync(hu, u, (size_t)n_edges * 4, cudaMemcpyHostToDevice, st));
        BBC_CUDA_TRY(cudaMemcpyAsync(hv, v, (size_t)n_edges * 4, cudaMemcpyHostToDevice, st));
        BBC_CUDA_TRY(cudaMemcpyAsync(hs, sign, (size_t)n_edges, cudaMemcpyHostToDevice, st));
        du = hu;
        dv = hv;
        ds = hs;
    }
    // 1. validate + degrees
    int32_t *deg_u = nullptr, *deg_v = nullptr;
    unsigned long long *stats = nullptr;  // [0] err, [1..2] U stats, [3..4] V stats, [5] dups
    BBC_TRY(sc.get(&deg_u, (size_t)n_u));
    BBC_TRY(sc.get(&deg_v, (size_t)n_v));
    BBC_TRY(sc.get(&stats, 8));
    if (n_u > 0) BBC_CUDA_TRY(cudaMemsetAsync(deg_u, 0, (size_t)n_u * 4, st));
    if (n_v > 0) BBC_CUDA_TRY(cudaMemsetAsync(deg_v, 0, (size_t)n_v * 4, st));
    BBC_CUDA_TRY(cudaMemsetAsync(stats, 0, 64, st));
    if (n_edges > 0) {
        note_launch();
        k_validate_degrees<<<grid_for(n_edges), kThreads, 0, st>>>(
            du, dv, ds, n_edges, n_u, n_v, deg_u, deg_v, reinterpret_cast<unsigned *>(stats));
        BBC_LAUNCH_CHECK("k_validate_degrees");
    }
    // 2. per-side sum of C(d,2) and max degree
    if (n_u > 0) {
        note_launch();
        k_degree_stats<<<grid_for(n_u), kThreads, 0, st>>>(deg_u, n_u, stats + 1);
        BBC_LAUNCH_CHECK("k_degree_stats");
    }
    if (n_v > 0) {
        note_launch();
        k_degree_stats<<<grid_for(n_v), kThreads, 0, st>>>(deg_v, n_v, stats + 3);
        BBC_LAUNCH_CHECK("k_degree_stats");
    }
    unsigned long long hst[8];
    BBC_CUDA_TRY(cudaMemcpyAsync(hst, stats, 64, cudaMemcpyDeviceToHost, st));
    BBC_CUDA_TRY(cudaStreamSynchronize(st));
    const unsigned err = (unsigned)(hst[0] & 0xffffffffu);
    if (err & 1u) {
        set_error("edge endpoint id out of range");
        return BBC_E_OUT_OF_RANGE;
    }
    if (err & 2u) {
        set_error("edge sign is not +1 or -1");
        return BBC_E_BAD_SIGN;
    }
    const uint64_t c2_u = hst[1], c2_v = hst[3];
    const int32_t max_u = (int32_t)hst[2], max_v = (int32_t)hst[4];
    // Pair side S: pairs on U visit sum_{v in V} C(d_v, 2) wedges, pairs on V visit
    // sum_{u in U} C(d_u, 2); the smaller wins (ties pick U).
    int side = c2_v <= c2_u ? 0 : 1;
    if (flags & BBC_SIDE_FORCE_U) side = 0;
    if (flags & BBC_SIDE_FORCE_V) side = 1;
    const int32_t nS = side == 0 ? n_u : n_v;
    const int32_t nC = side == 0 ? n_v : n_u;
    const int32_t *degS = side == 0 ? deg_u : deg_v;
    const int32_t *degC = side == 0 ? deg_v : deg_u;
    const int32_t maxS = side == 0 ? max_u : max_v;
    const int32_t maxC = side == 0 ? max_v : max_u;
    const uint64_t W = side == 0 ? c2_v : c2_u;
    {
        // balanced <= sum over pairs of C(c, 2) <= W * (max degree on S - 1) / 2
        const unsigned __int128 bound = (unsigned __int128)W * (unsigned)(maxS > 0 ? maxS - 1 : 0) / 2;
        if (bound > (unsigned __int128)UINT64_MAX) {
            set_error("counts may exceed 2^64 - 1");
            return BBC_E_OVERFLOW_RISK;
        }
    }

    bbc_graph *g = new (std::nothrow) bbc_graph();
    if (!g) {
        set_error("host allocation failed");
        return BBC_E_NO_MEMORY;
    }
    struct Guard {
        bbc_graph *g;
        cudaStream_t st;
        ~Guard() {
            if (g) release_graph(g, st);
        }
    } guard{g, st};
    static std::atomic<uint64_t> next_uid{1};
    g->uid = next_uid.fetch_add(1);
    cudaGetDevice(&g->device);
    g->n_u = n_u;
    g->n_v = n_v;
    g->side = side;
    g->side_paper_rule = n_v < n_u ? 1 : 0;
    g->orient_low = (flags & BBC_ORIENT_LOW_ANCHOR) ? 1 : 0;
    g->nS = nS;
    g->nC = nC;
    g->wedges = W;
    g->max_deg_S = maxS;
    g->max_deg_C = maxC;

    // 3. ranks
    int32_t *rankS = nullptr, *rankC = nullptr;
    BBC_TRY(sc.get(&rankS, (size_t)nS));
    BBC_TRY(sc.get(&rankC, (size_t)nC));
    BBC_TRY(dev_alloc_n(&g->permS, (size_t)nS, st));
    BBC_TRY(dev_alloc_n(&g->permC, (size_t)nC, st));
    BBC_TRY(rank_side(degS, nS, maxS, rankS, g->permS, st));
    BBC_TRY(rank_side(degC, nC, maxC, rankC, g->permC, st));

    // 4. the two CSR arrays
    const int64_t E = n_edges;
    uint32_t *kA = nullptr, *vA = nullptr, *kB = nullptr, *vB = nullptr;
    BBC_TRY(dev_alloc_n(&kA, (size_t)E, st));   // becomes g->anchor_of after the sort
    g->anchor_of = kA;
    BBC_TRY(dev_alloc_n(&vA, (size_t)E, st));
    g->rowS = vA;
    BBC_TRY(sc.get(&kB, (size_t)E));
    BBC_TRY(dev_alloc_n(&vB, (size_t)E, st));
    g->rowC = vB;
    if (E > 0) {
        note_launch();
        k_map_edges<<<grid_for(E), kThreads, 0, st>>>(du, dv, ds, E, side, rankS, rankC, kA, vA);
        BBC_LAUNCH_CHECK("k_map_edges");
        BBC_TRY(radix_sort_pairs(kA, vA, E, bit_length((uint64_t)(nS > 0 ? nS - 1 : 0)), st));
        note_launch();
        k_swap_sides<<<grid_for(E), kThreads, 0, st>>>(kA, vA, E, kB, vB);
        BBC_LAUNCH_CHECK("k_swap_sides");
        BBC_TRY(radix_sort_pairs(kB, vB, E, bit_length((uint64_t)(nC > 0 ? nC - 1 : 0)), st));
        note_launch();
        k_count_duplicates<<<grid_for(E), kThreads, 0, st>>>(kB, vB, E, stats + 5);
        BBC_LAUNCH_CHECK("k_count_duplicates");
        unsigned long long dups = 0;
        BBC_CUDA_TRY(cudaMemcpyAsync(&dups, stats + 5, 8, cudaMemcpyDeviceToHost, st));
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        if (dups) {
            if (!(flags & BBC_DEDUP_LAST)) {
                set_error("duplicate (u, v) pair in the edge list");
                return BBC_E_DUPLICATE_EDGE;
            }
            // Keep the last occurrence of each pair and prepare the de-duplicated list.
            int32_t *flag = nullptr;
            int64_t *pos = nullptr;
            BBC_TRY(sc.get(&flag, (size_t)E));
            BBC_TRY(sc.get(&pos, (size_t)E + 1));
            note_launch();
            k_last_flags<<<grid_for(E), kThreads, 0, st>>>(kB, vB, E, flag);
            BBC_LAUNCH_CHECK("k_last_flags");
            BBC_TRY(exclusive_scan_i32_to_i64(flag, pos, E, st));
            const int64_t E2 = E - (int64_t)dups;
            int32_t *u2 = nullptr, *v2 = nullptr;
            int8_t *s2 = nullptr;
            BBC_TRY(sc.get(&u2, (size_t)E2));
            BBC_TRY(sc.get(&v2, (size_t)E2));
            BBC_TRY(sc.get(&s2, (size_t)E2));
            note_launch();
            k_dedup_last<<<grid_for(E), kThreads, 0, st>>>(kB, vB, E, pos, side, g->permS, g->permC,
                                                            u2, v2, s2);
            BBC_LAUNCH_CHECK("k_dedup_last");
            return prepare_graph(n_u, n_v, E2, u2, v2, s2,
                                 (flags | BBC_INPUT_DEVICE) & ~(uint32_t)BBC_DEDUP_LAST, st, out);
        }
    }
    g->n_edges = E;

    // 5. row offsets from the ranked degrees
    int32_t *dr = nullptr;
    BBC_TRY(sc.get(&dr, (size_t)std::max(nS, nC)));
    BBC_TRY(dev_alloc_n(&g->rowS_off, (size_t)nS + 1, st));
    BBC_TRY(dev_alloc_n(&g->rowC_off, (size_t)nC + 1, st));
    if (nS > 0) {
        note_launch();
        k_gather_deg<<<grid_for(nS), kThreads, 0, st>>>(degS, g->permS, nS, dr);
        BBC_LAUNCH_CHECK("k_gather_deg");
    }
    BBC_TRY(exclusive_scan_i32_to_i64(dr, g->rowS_off, nS, st));
    if (nC > 0) {
        note_launch();
        k_gather_deg<<<grid_for(nC), kThreads, 0, st>>>(degC, g->permC, nC, dr);
        BBC_LAUNCH_CHECK("k_gather_deg");
    }
    BBC_TRY(exclusive_scan_i32_to_i64(dr, g->rowC_off, nC, st));

    // 6. oriented wedges per anchor
    BBC_TRY(dev_alloc_n(&g->wl, (size_t)nS, st));
    BBC_TRY(dev_alloc_n(&g->rng, (size_t)E, st));
    if (nS > 0) BBC_CUDA_TRY(cudaMemsetAsync(g->wl, 0, (size_t)nS * 8, st));
    if (E > 0) {
        note_launch();
        k_wedge_estimate<<<grid_for(E), kThreads, 0, st>>>(kA, g->rowS, E, g->rowC_off, g->rowC,
                                                             g->orient_low, g->wl, g->rng);
        BBC_LAUNCH_CHECK("k_wedge_estimate");
    }
    BBC_TRY(dev_alloc_n(&g->totals, 2, st));
    BBC_TRY(dev_alloc_n(&g->queue, 1, st));
    BBC_TRY(dev_alloc_n(&g->dgraph, 1, st));
    g->device_bytes = (size_t)(nS + 1 + nC + 1) * 8 + (size_t)E * 20 + (size_t)(nS + nC) * 4 +
                      (size_t)nS * 8;
    *out = g;
    guard.g = nullptr;
    return BBC_OK;
}

}  // namespace bbc
