// count.cu -- the counting kernels (bbc_count's hot path).
//
// For an anchor a of the pair side S, every oriented wedge a - c - w (c a centre
// neighbour of a, w an endpoint of higher rank than a) is bucketed by its endpoint w and
// its type: symmetric when the two edge signs agree (Def. 8), asymmetric otherwise
// (Def. 9). Once every wedge of a has been bucketed, endpoint w closes C(p,2) + C(n,2)
// balanced butterflies with a (Lemma 1), where p / n are its two counters. This is the
// B1/B2 bucket scheme of BB2K (Algorithm 1) and G-BBC (Algorithm 3), laid out for
// sm_103a:
//
//   * k_tile: persistent blocks pop (anchor, tile range) items from an atomic queue
//     (the dynamic scheduling of G-BBC++, Algorithm 4). A tile is a dense shared-memory
//     counter array over a window of endpoint ranks (Fig. 4's tiles), with two 8-, 16-
//     or 32-bit counters per endpoint. The width is chosen tile by tile, since a tile's
//     first endpoint bounds its counts. Each C -> S row is sorted by rank, so the wedges
//     of centre c in the window are one contiguous slice. Per chunk of 512 centres, the
//     short slices are swept by warps with lanes on consecutive positions, and the long
//     ones in 1,024-wedge pieces with 16-byte loads.
//     An anchor too heavy for its tiles to spread over the blocks has each tile's
//     centres cut into parts whose counts merge in device memory; with per-vertex
//     output, k_tile_cs then runs those parts' centre passes.
//   * k_group_tile<4> / k_group_tile<1>: anchors whose whole endpoint range fits a
//     4-warp group's or one warp's table.
//   * k_warp_hash: light anchors (few wedges) get one warp each and a small open-
//     addressing hash table in shared memory, so their cost follows their wedge count
//     and not the width of their endpoint range.
//   * k_tile_motif: the same sweep with the counters and epilogue of the sign classes
//     (Sec. VII) or of balanced (2,k)-bicliques (Def. 5).
//
// Per-vertex counts (an extension: the paper defines none) follow from the same
// counters: the pair {a, w} adds f = C(p,2) + C(n,2) to both b(a) and b(w); and a wedge
// a - c - w of type t lies in (count_t(a, w) - 1) balanced butterflies through c, so a
// second sweep over the same slices, after the counters are complete, adds that to b(c).
#include <algorithm>
#include <climits>
#include <type_traits>

#include "graph.cuh"

namespace bbc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTileThreads = 512;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kChunk = kTileThreads;      // centres per block-sweep chunk
constexpr int kLongMin = 64;              // slices this long are cut into pieces
// the chunk scan packs a chunk's short-slice wedges into 16 bits
static_assert((kLongMin - 1) * kChunk < (1 << 16), "short-slice wedges of a chunk exceed the scan field");
constexpr int kPiece = 1024;              // wedges per piece of a long slice
// how the tile kernel's blocks take items: rank order by block index (Algorithm 3's static
// mapping), the atomic queue, or the queue with the next item taken one item early
enum { kScheduleQueue = 0, kScheduleStatic = 1, kScheduleQueueAhead = 2 };
constexpr int kLongSlice = 64;            // warp sweep: slices this long use the whole warp
constexpr int kWtThreads = 512;          // warp-tile kernel: 16 warps, one table each
constexpr int kWtWarps = kWtThreads / 32;
constexpr int kHashThreads = 256;
constexpr int kHashWarps = kHashThreads / 32;
constexpr int kHashSlots = 1024;          // most per warp; holds anchors of <= 512 wedges
constexpr uint32_t kEmpty = 0xffffffffu;

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

// Fire-and-forget 64-bit add to global memory. The per-vertex and total counters are
// reached through pointers loaded from the graph descriptor, which the compiler cannot
// place in the global space, so atomicAdd there becomes a generic atomic that waits for
// its old value; the explicit reduction does not.
__device__ __forceinline__ void red_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v) : "memory");
}

// A hint that brings a line of global memory into L2 (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

__device__ __forceinline__ unsigned long long choose2(unsigned long long x) {
    return x * (x - (x > 0)) / 2;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// ----------------------------------------------------------------------------- counters

// Open addressing (linear probing) over `mask + 1` slots; values are packed p | n << 16.
// The table is sized to at least twice the anchor's wedge count, so it never fills; the
// probe loops are still bounded and report kErrHashFull instead of spinning.
struct HashCounter {
    uint32_t *keys;
    uint32_t *vals;
    uint32_t mask;
    int shift;
    unsigned *err;
    __device__ __forceinline__ uint32_t home(uint32_t w) const { return (w * 0x9E3779B1u) >> shift; }
    __device__ __forceinline__ void bump(uint32_t w, uint32_t t) const {
        volatile uint32_t *vk = keys;
        uint32_t h = home(w);
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            const uint32_t k = vk[h];
            if (k == w) {
                atomicAdd(vals + h, 1u << (t << 4));
                return;
            }
            if (k == kEmpty) {
                const uint32_t old = atomicCAS(keys + h, kEmpty, w);
                if (old == kEmpty || old == w) {
                    atomicAdd(vals + h, 1u << (t << 4));
                    return;
                }
            }
            h = (h + 1) & mask;
        }
        atomicOr(err, kErrHashFull);
    }
    __device__ static __forceinline__ uint32_t sign_key(uint32_t sg) { return sg; }
    __device__ __forceinline__ void bump_entry(uint32_t x, uint32_t sg) const { bump(x & kIdMask, (x ^ sg) >> 31); }
    __device__ __forceinline__ uint32_t count_entry(uint32_t x, uint32_t sg) const {
        return peek(x & kIdMask, (x ^ sg) >> 31);
    }
    __device__ __forceinline__ uint32_t peek(uint32_t w, uint32_t t) const {
        uint32_t h = home(w);
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            const uint32_t k = keys[h];
            if (k == w) return (vals[h] >> (t << 4)) & 0xffffu;
            if (k == kEmpty) break;
            h = (h + 1) & mask;
        }
        atomicOr(err, kErrHashFull);
        return 1u;
    }
};

// ----------------------------------------------------------------------------- sweep

// ----------------------------------------------------------------------------- tiles

// Dense counters over the endpoint ranks [lo, lo + endpoints) of one tile. The counter
// width follows the largest count the anchor can reach (its degree, or its wedge count
// if smaller): CW 0 packs two endpoints of two 8-bit counters (p, n) per word, CW 1 one
// endpoint of two 16-bit counters, CW 2 one endpoint of two 32-bit words.
template <int CW>
struct TileCounter {
    uint32_t *tile;
    uint32_t lo;
    __device__ __forceinline__ void bump(uint32_t w, uint32_t t) const {
        const uint32_t e = w - lo;
        if (CW == 0)
            atomicAdd(tile + (e >> 1), 1u << (((e & 1u) << 4) | (t << 3)));
        else if (CW == 1)
            atomicAdd(tile + e, 1u << (t << 4));
        else
            atomicAdd(tile + 2 * e + t, 1u);
    }
    __device__ __forceinline__ uint32_t peek(uint32_t w, uint32_t t) const {
        const uint32_t e = w - lo;
        if (CW == 0) return (tile[e >> 1] >> (((e & 1u) << 4) | (t << 3))) & 0xffu;
        if (CW == 1) return (tile[e] >> (t << 4)) & 0xffffu;
        return tile[2 * e + t];
    }
    // a C -> S entry x (endpoint rank | sign << 31) reached through an anchor edge of
    // sign bit sg: the wedge is symmetric (t = 0) or asymmetric (t = 1)
    __device__ static __forceinline__ uint32_t sign_key(uint32_t sg) { return sg; }
    __device__ __forceinline__ void bump_entry(uint32_t x, uint32_t sg) const {
        bump(x & kIdMask, (x ^ sg) >> 31);
    }
    __device__ __forceinline__ uint32_t count_entry(uint32_t x, uint32_t sg) const {
        return peek(x & kIdMask, (x ^ sg) >> 31);
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void smem_red_add(uint32_t a, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v));
}
__device__ __forceinline__ uint32_t smem_load(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t rotl(uint32_t x, int k) { return __funnelshift_l(x, x, k); }

// The block tile of k_tile, the same counters as TileCounter's but addressed through
// 32-bit shared-memory addresses with the tile's origin folded into one base, so that a
// C -> S entry x (endpoint rank w | sign << 31) reaches its counter in a few integer
// operations. Byte offset of the counter of endpoint w and wedge type t:
//   CW 0: 2 (w - org) + t with org = lo rounded down to even (a word holds the counters
//         of an even and an odd endpoint: bytes p0, n0, p1, n1);
//   CW 1: 4 (w - org) + 2 t with org = lo;
//   CW 2: 8 (w - org) + 4 t with org = lo.
// The counter's index 2 w + t is x xor the anchor edge's sign bit, rotated left by one,
// so the centre pass loads each counter at its own width from base + width * that. The
// count pass needs word-sized atomics: the word is (base + 2x) & ~3 (CW 0) or base + 4x
// (CW 1), and the counter's bit offset in it, 16 (w & 1) + 8 t (CW 0) or 16 t (CW 1), is
// x's low bit and sign bit brought into place by one rotation, with the anchor edge's
// sign xor-ed in.
// All address arithmetic is modulo 2^32, so bits shifted out of x (its sign, and high
// rank bits) only add multiples of 2^32 and the address stays exact. A tile whose lo is
// odd uses one word beyond tile_words with 8-bit counters (the kernel allocates it).
template <int CW>
struct BlockTile {
    uint32_t base;
    __device__ static __forceinline__ uint32_t origin(uint32_t lo) { return CW == 0 ? (lo & ~1u) : lo; }
    __device__ __forceinline__ BlockTile(const uint32_t *tile, uint32_t lo) {
        const uint32_t a = smem_addr(tile), o = origin(lo);
        base = a - (CW == 0 ? 2u : (CW == 1 ? 4u : 8u)) * o;
    }
    // the anchor edge's sign bit, as the slice's key
    __device__ static __forceinline__ uint32_t sign_key(uint32_t sg) { return sg; }
    // the word holding the counter (atomics are word-sized)
    __device__ __forceinline__ uint32_t word(uint32_t x, uint32_t sk) const {
        if (CW == 0) return (base + 2u * x) & ~3u;
        if (CW == 1) return base + 4u * x;
        return base + 4u * rotl(x ^ sk, 1);
    }
    // the counter's bit offset within that word (the sign keys shifted into place are
    // loop invariants of a slice)
    __device__ __forceinline__ uint32_t shift(uint32_t x, uint32_t sk) const {
        if (CW == 0) return (rotl(x, 4) ^ (sk >> 28)) & 24u;
        if (CW == 1) return (rotl(x, 5) ^ (sk >> 27)) & 16u;
        return 0u;
    }
    // the counter's own address: rotl(x ^ sg, 1) is 2 w + t, the counter's index
    __device__ __forceinline__ uint32_t counter(uint32_t x, uint32_t sk) const {
        return base + (CW == 0 ? 1u : (CW == 1 ? 2u : 4u)) * rotl(x ^ sk, 1);
    }
    __device__ __forceinline__ void bump_entry(uint32_t x, uint32_t sk) const {
        smem_red_add(word(x, sk), CW == 2 ? 1u : 1u << shift(x, sk));
    }
    // the counter of the wedge's endpoint and type (its full count, once the tile is done),
    // read at its own width
    __device__ __forceinline__ uint32_t count_entry(uint32_t x, uint32_t sk) const {
        const uint32_t a = counter(x, sk);
        uint32_t v;
        if (CW == 0)
            asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
        else if (CW == 1)
            asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
        else
            v = smem_load(a);
        return v;
    }
    __device__ __forceinline__ void add_count(uint32_t x, uint32_t sk, uint32_t &acc) const {
        acc += count_entry(x, sk);
    }
    __device__ __forceinline__ void add_count(uint32_t x, uint32_t sk, unsigned long long &acc) const {
        acc += count_entry(x, sk);
    }
};

// Sign-class counters (Sec. VII): per endpoint the centres whose two edges are both +
// (kind 0), both - (kind 1), or of different signs (kind 2). CW 0: one word of bytes
// (pp, nn, a, 0); CW 1: two words (pp | nn << 16, a); CW 2: four 32-bit words. An
// endpoint takes twice the words of TileCounter's layout.
template <int CW>
struct ClassCounter {
    uint32_t *tile;
    uint32_t lo;
    __device__ __forceinline__ void bump_entry(uint32_t x, uint32_t sg) const {
        const uint32_t e = (x & kIdMask) - lo;
        const uint32_t kind = ((x ^ sg) >> 31) ? 2u : (sg >> 31);
        if (CW == 0)
            atomicAdd(tile + e, 1u << (kind << 3));
        else if (CW == 1)
            atomicAdd(tile + 2 * e + (kind >> 1), kind == 2 ? 1u : 1u << (kind << 4));
        else
            atomicAdd(tile + 4 * e + kind, 1u);
    }
    __device__ static __forceinline__ uint32_t sign_key(uint32_t sg) { return sg; }
    __device__ __forceinline__ uint32_t count_entry(uint32_t, uint32_t) const { return 1u; }
    template <class A>
    __device__ __forceinline__ void add_count(uint32_t, uint32_t, A &acc) const { acc += 1u; }
    __device__ __forceinline__ void read(uint32_t e, uint32_t &pp, uint32_t &nn, uint32_t &a) const {
        if (CW == 0) {
            const uint32_t v = tile[e];
            pp = v & 0xffu;
            nn = (v >> 8) & 0xffu;
            a = (v >> 16) & 0xffu;
        } else if (CW == 1) {
            const uint32_t v = tile[2 * e];
            pp = v & 0xffffu;
            nn = v >> 16;
            a = tile[2 * e + 1];
        } else {
            pp = tile[4 * e];
            nn = tile[4 * e + 1];
            a = tile[4 * e + 2];
        }
    }
    static constexpr uint32_t words_per_endpoint = CW == 0 ? 1u : (CW == 1 ? 2u : 4u);
};

__host__ __device__ constexpr uint32_t endpoints_per_tile(int cw, uint32_t tile_words) {
    return cw == 0 ? tile_words * 2 : (cw == 1 ? tile_words : tile_words / 2);
}

// Per-chunk bookkeeping of the block sweep: the slice of every centre of the chunk and
// two prefix sums, over short-slice wedges and over long-slice pieces.
struct ChunkSmem {
    uint32_t ent[kChunk];
    uint32_t start[kChunk];
    uint32_t len[kChunk];
    uint32_t ppiece[kChunk + 1];
    // the chunk's non-empty short slices, compacted in centre order: concatenated start
    // (sP[nz] = ns, the chunk's short-wedge total), rowC index minus that start, and the
    // centre's sign bit | its index in the chunk
    uint32_t sP[kChunk + 1];
    uint32_t sbase[kChunk];
    uint32_t smeta[kChunk];
    unsigned long long acc[kChunk];
    unsigned long long wsum[kTileWarps];
    uint32_t ns, nz;
};
// index of the last entry <= k in the non-decreasing p[0..n] (p[0] == 0 <= k)
__device__ __forceinline__ int last_le_n(const uint32_t *p, int n, uint32_t k) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p[mid] <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long block_exclusive_scan_u64(unsigned long long x,
                                                                      unsigned long long &total,
                                                                      unsigned long long *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    // every warp scans the warp sums itself (no second barrier)
    const unsigned long long w = lane < kTileWarps ? wsum[lane] : 0ull;
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < kTileWarps; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += y;
    }
    total = __shfl_sync(kFull, wi, kTileWarps - 1);
    return __shfl_sync(kFull, wi - w, warp) + inc - x;
}

// Per-wedge work. MODE 1 sums (count - 1); with 8- and 16-bit counters a thread's or a
// piece's sum stays far below 2^32 (at most 1,024 wedges of count <= 65,535), so it is
// kept in 32 bits; 32-bit counters use 64-bit sums.
template <int CW>
using Acc = typename std::conditional<CW == 2, unsigned long long, uint32_t>::type;


// One wedge given by its C -> S entry x and the counter's sign key of the anchor edge:
// MODE 0 bumps its counter; MODE 1 adds the counter's value to acc (the caller subtracts
// one per wedge afterwards).
template <int MODE, int CW, class Ctr>
__device__ __forceinline__ void wedge(const Ctr &ctr, uint32_t x, uint32_t sk, Acc<CW> &acc) {
    if constexpr (MODE == 0)
        ctr.bump_entry(x, sk);
    else
        ctr.add_count(x, sk, acc);
}

// Sum over a warp of a per-lane accumulator (one redux instruction for 32 bits).
__device__ __forceinline__ uint32_t warp_total(uint32_t x) { return __reduce_add_sync(kFull, x); }
__device__ __forceinline__ unsigned long long warp_total(unsigned long long x) { return warp_sum(x); }

// One wedge for any counter and accumulator type (wedge() without the width).
template <int MODE, class Ctr, class A>
__device__ __forceinline__ void wedge_any(const Ctr &ctr, uint32_t x, uint32_t sk, A &acc) {
    if constexpr (MODE == 0)
        ctr.bump_entry(x, sk);
    else
        acc += ctr.count_entry(x, sk);
}

// Lane-interleaved walk over positions [r0, r1) of a run of concatenated short slices, 32
// consecutive positions per step with lane L on position r + L, so that lanes on one
// slice read consecutive entries (coalesced). sP[0..nz] are the slices' starts in the
// concatenation (strictly increasing; sP[nz] is the total), sbase[j] is the rowC index of
// slice j's first entry minus sP[j], and smeta[j] holds the anchor edge's sign bit and a
// tag below 2^31. A lane's slice is the window's first slice plus the number of slice
// starts at or before its position, counted from a bit mask of the starts inside the
// window. The entries of the next AHEAD (1 or 2) windows are loaded before this window's
// counters are touched, so AHEAD + 1 loads per lane are in flight. MODE 1 hands each run
// of lanes on one slice, once per window, to add(tag, sum over its wedges of count - 1).
template <int MODE, class A, int AHEAD, class Ctr, class Add>
__device__ __forceinline__ void walk_short(const Ctr &ctr, const uint32_t *__restrict__ rowC,
                                           const uint32_t *sP, const uint32_t *sbase,
                                           const uint32_t *smeta, int nz, uint32_t r0, uint32_t r1,
                                           Add &&add) {
    const int lane = threadIdx.x & 31;
    // window r: each lane's slice (-1 past r1), the bit mask of the slices that start
    // inside the window (set bit d: a slice starts at r + d; the starts of the up to 32
    // slices after jbase all lie past r), and the slice at position r + 32
    auto locate = [&](uint32_t r, int jbase, uint32_t &m, int &j, int &jnext) {
        const int jl = jbase + 1 + lane;
        const uint32_t e = jl <= nz ? sP[jl] : 0xffffffffu;
        const uint32_t d = e - r;
        m = __reduce_or_sync(kFull, d < 32u ? 1u << d : 0u);
        const bool at32 = __any_sync(kFull, d == 32u);
        j = r + (uint32_t)lane < r1 ? jbase + __popc(m & ((2u << lane) - 1u)) : -1;
        jnext = jbase + __popc(m) + (at32 ? 1 : 0);
    };
    // one window's slice mask, lane slice, sign/tag and entry, loaded AHEAD windows
    // before it is used
    struct Stage {
        uint32_t m = 0, x = 0, meta = 0;
        int j = -1;
    };
    auto fetch = [&](uint32_t r, int jbase, Stage &st, int &jnext) {
        st = Stage{};
        jnext = jbase;
        if (r < r1) {
            locate(r, jbase, st.m, st.j, jnext);
            if (st.j >= 0) {
                st.meta = smeta[st.j];
                st.x = __ldg(rowC + (uint32_t)(sbase[st.j] + r + lane));
            }
        }
    };
    Stage s0, s1, s2;
    int jn = 0;
    fetch(r0, last_le_n(sP, nz, r0), s0, jn);
    if (AHEAD == 2) fetch(r0 + 32u, jn, s1, jn);
    for (uint32_t r = r0; r < r1; r += 32u) {
        if (AHEAD == 2)
            fetch(r + 64u, jn, s2, jn);
        else
            fetch(r + 32u, jn, s1, jn);
        const uint32_t m = s0.m, x = s0.x, meta = s0.meta;
        const int j = s0.j;
        A v = 0;
        if (j >= 0) {
            wedge_any<MODE>(ctr, x, Ctr::sign_key(meta & kSignBit), v);
            if (MODE == 1) v -= 1u;
        }
        if constexpr (MODE == 1 && sizeof(A) == 4) {
            // lanes of one slice are contiguous and a new slice starts at every set bit of
            // m: each lane's group is the run of lanes between two such bits, summed by
            // one redux; its first lane hands the sum on
            const uint32_t upto = (2u << lane) - 1u;
            const int g0 = 31 - __clz((m & upto) | 1u);
            const uint32_t above = m & ~upto;
            const uint32_t hi_mask = above ? (above & (0u - above)) - 1u : kFull;
            const uint32_t gmask = hi_mask & ~((1u << g0) - 1u);
            const uint32_t tot = __reduce_add_sync(gmask, (uint32_t)v);
            if (lane == g0 && j >= 0 && tot) add(meta & kIdMask, (A)tot);
        } else if constexpr (MODE == 1) {
            // segmented sum over lanes of the same slice; the last lane of each hands it on
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const A y = __shfl_up_sync(kFull, v, o);
                const int jj = __shfl_up_sync(kFull, j, o);
                if (lane >= o && jj == j) v += y;
            }
            const int jnb = __shfl_down_sync(kFull, j, 1);
            if (j >= 0 && (lane == 31 || jnb != j) && v) add(meta & kIdMask, v);
        }
        s0 = s1;
        if (AHEAD == 2) s1 = s2;
    }
}

// Per-warp staging of one batch of 32 centres' short slices (the warp sweep's table):
// the compacted non-empty short slices in lane order, as walk_short reads them.
struct WarpStage {
    uint32_t sP[33];
    uint32_t sbase[32];
    uint32_t meta[32];
};

// One warp's pass over all oriented wedges of anchor rows [sb, se) (the warp kernels'
// sweep: their anchors fit one counter table). MODE 0 bumps the counters; MODE 1 (the
// per-vertex centre pass) reads them and adds (count - 1) per wedge to the centre's b.
// Warps take batches of `batch` (<= 32) centres from *batch_ctr (or, with batch_ctr NULL,
// one warp takes them all in order); lane j owns centre j's slice. Long
// slices are swept by the whole warp with 16-byte loads; short ones are compacted into
// the warp's stage and walked lane-interleaved (walk_short, AHEAD windows loaded ahead:
// the hash kernel keeps one for its registers). Per-centre sums of a batch stay below
// 2^32: a slice's counts add up to at most the number of edges.
template <int MODE, int AHEAD = 2, class Counter>
__device__ __forceinline__ void warp_sweep(const DevGraph &G, int64_t sb, int64_t se,
                                      const Counter &ctr, int *batch_ctr, uint32_t *sacc,
                                      WarpStage &ws, int batch = 32) {
    const int lane = threadIdx.x & 31;
    const int64_t nbatch = (se - sb + batch - 1) / batch;
    int next_private = 0;   // a warp alone on its anchor (batch_ctr NULL) takes every batch
    const uint32_t *__restrict__ rowC = G.rowC;
    for (;;) {
        int bi = next_private++;
        if (batch_ctr) {
            if (lane == 0) bi = atomicAdd(batch_ctr, 1);
            bi = __shfl_sync(kFull, bi, 0);
        }
        if (bi >= nbatch) break;
        const int64_t ci = sb + (int64_t)bi * batch + lane;
        uint32_t b = 0, len = 0, sg = 0, c = 0;
        if (lane < batch && ci < se) {
            // the whole endpoint range of the anchor inside row c (known from preparation)
            const uint32_t ent = __ldg(G.rowS + ci);
            c = ent & kIdMask;
            sg = ent & kSignBit;
            const uint2 r = __ldg(G.rng + ci);
            b = r.x;
            len = r.y - r.x;
        }
        // Long slices: the whole warp sweeps one slice at a time, coalesced 16-byte loads.
        unsigned longm = __ballot_sync(kFull, len >= (uint32_t)kLongSlice);
        while (longm) {
            const int j = __ffs(longm) - 1;
            longm &= longm - 1;
            const uint32_t s = __shfl_sync(kFull, b, j);
            const uint32_t n = __shfl_sync(kFull, len, j);
            const uint32_t sj = Counter::sign_key(__shfl_sync(kFull, sg, j));
            uint32_t acc = 0;
            auto visit = [&](uint32_t x) {
                if (MODE == 0)
                    ctr.bump_entry(x, sj);
                else
                    acc += ctr.count_entry(x, sj);
            };
            const uint32_t head = min(n, (4u - (s & 3u)) & 3u);
            if ((uint32_t)lane < head) visit(__ldg(rowC + s + lane));
            const uint32_t m4 = (n - head) >> 2;
            const uint4 *v4 = reinterpret_cast<const uint4 *>(rowC + s + head);
            for (uint32_t q = lane; q < m4; q += 64) {
                const uint4 xa = __ldg(v4 + q);
                const bool has_b = q + 32 < m4;
                uint4 xb = make_uint4(0u, 0u, 0u, 0u);
                if (has_b) xb = __ldg(v4 + q + 32);
                visit(xa.x);
                visit(xa.y);
                visit(xa.z);
                visit(xa.w);
                if (has_b) {
                    visit(xb.x);
                    visit(xb.y);
                    visit(xb.z);
                    visit(xb.w);
                }
            }
            const uint32_t rest = (n - head) & 3u;
            if ((uint32_t)lane < rest) visit(__ldg(rowC + s + head + 4 * m4 + lane));
            if (MODE == 1) {
                const uint32_t tot = warp_total(acc) - n;
                if (lane == j && tot) red_add(G.bC + c, tot);
            }
        }
        // Short slices: compacted in lane order, then walked lane-interleaved.
        const bool isshort = len > 0 && len < (uint32_t)kLongSlice;
        const unsigned smask = __ballot_sync(kFull, isshort);
        const uint32_t sl = isshort ? len : 0u;
        uint32_t incl = sl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        const int nzs = __popc(smask);
        if (isshort) {
            const int cj = __popc(smask & ((1u << lane) - 1u));
            ws.sP[cj] = incl - sl;
            ws.sbase[cj] = b - (incl - sl);
            ws.meta[cj] = sg | (uint32_t)lane;
        }
        if (lane == 0) ws.sP[nzs] = total;
        if (MODE == 1) sacc[lane] = 0;
        __syncwarp();
        if (total)
            walk_short<MODE, uint32_t, AHEAD>(ctr, rowC, ws.sP, ws.sbase, ws.meta, nzs, 0u, total,
                                       [&](uint32_t tag, uint32_t v) { atomicAdd(sacc + tag, v); });
        __syncwarp();
        if (MODE == 1) {
            if (isshort && sacc[lane]) red_add(G.bC + c, sacc[lane]);
            __syncwarp();
        }
    }
}

// First index of row[b, lim) whose rank is >= key (the row is sorted by rank), found by
// galloping from b: about 2 log2 of the distance instead of log2 of the row length.
__device__ __forceinline__ uint32_t gallop_rank(const uint32_t *__restrict__ row, uint32_t b,
                                                uint32_t lim, uint32_t key) {
    uint32_t lo = b, step = 1;
    while (lo + step <= lim && (__ldg(row + lo + step - 1) & kIdMask) < key) {
        lo += step;
        step <<= 1;
    }
    uint32_t hi = min(lo + step - 1, lim);
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if ((__ldg(row + m) & kIdMask) < key)
            lo = m + 1;
        else
            hi = m;
    }
    return lo;
}

// Where one tile's slices come from.
struct SweepCtx {
    uint32_t lo, hi;              // the tile's endpoint ranks [lo, hi)
    uint32_t range_lo, range_hi;  // the anchor's whole endpoint range
    int t, nt;                    // this tile, and the anchor's number of tiles
    int64_t bbase;                // boff[anchor]
    int64_t deg;                  // the anchor's degree
    int64_t row0;                 // the anchor's first S -> C entry
    bool single;                  // all centres fit one chunk: slices stay in shared memory
};

// The slice of row c (entry e, the i-th of the anchor's S -> C row) whose endpoint ranks
// lie in [X.lo, X.hi). The anchor's whole range inside row c is known from preparation
// (rng), so the first tile starts and the last ends there; interior boundaries come from
// the table computed with the work lists (bnd), or, without it, from a binary search and
// a gallop.
__device__ __forceinline__ void find_slice(const DevGraph &G, int64_t e, int64_t i,
                                           const SweepCtx &X, uint32_t &start, uint32_t &len) {
    const uint2 r = __ldg(G.rng + e);
    uint32_t b, en;
    if (G.bnd) {
        b = X.t == 0 ? r.x : __ldg(G.bnd + X.bbase + (int64_t)(X.t - 1) * X.deg + i);
        en = X.t == X.nt - 1 ? r.y : __ldg(G.bnd + X.bbase + (int64_t)X.t * X.deg + i);
    } else {
        b = X.t == 0 ? r.x : (uint32_t)lower_bound_rank(G.rowC, r.x, r.y, X.lo);
        en = X.t == X.nt - 1 ? r.y : gallop_rank(G.rowC, b, min(r.y, b + (X.hi - X.lo)), X.hi);
    }
    start = b;
    len = en - b;
}

// Adds a chunk-centre's per-tile sum into the chunk accumulator (cs.acc, read as 32-bit
// words for 8- and 16-bit counters: a centre's sum over one tile is at most 25,176
// endpoints times 65,534 < 2^32).
template <int CW>
__device__ __forceinline__ void acc_add(ChunkSmem &cs, int j, Acc<CW> v) {
    if (CW == 2)
        atomicAdd(cs.acc + j, (unsigned long long)v);
    else
        atomicAdd(reinterpret_cast<uint32_t *>(cs.acc) + j, (uint32_t)v);
}

template <int CW>
__device__ __forceinline__ unsigned long long acc_get(ChunkSmem &cs, int j) {
    return CW == 2 ? cs.acc[j] : (unsigned long long)reinterpret_cast<uint32_t *>(cs.acc)[j];
}

// One pass of the whole block over the oriented wedges of anchor rows [sb, se) whose
// endpoints lie in [X.lo, X.hi), in chunks of kChunk centres. Per chunk, every thread
// finds its centre's slice; slices shorter than kLongMin are concatenated and cut into
// equal contiguous shares, one per warp, read 32 consecutive positions at a time; longer
// ones are cut into kPiece-wedge pieces that the warps take round robin and sweep with
// coalesced 16-byte loads. MODE 0
// bumps the counters; MODE 1 reads them and adds (count - 1) per wedge to the centre's
// per-vertex sum. A single-chunk MODE 1 pass reuses the slices MODE 0 just found.
template <int MODE, int CW, class Ctr, bool PF = false>
__device__ void block_sweep(const DevGraph &G, int64_t sb, int64_t se, const SweepCtx &X,
                            const Ctr &ctr, ChunkSmem &cs, unsigned long long &centre_carry) {
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t *__restrict__ rowC = G.rowC;
    for (int64_t cb = sb; cb < se; cb += kChunk) {
        const int64_t ci = cb + tid;
        uint32_t ent = 0;
        if (MODE == 1 && X.single) {
            // the count pass of this tile found the slices, zeroed the accumulators and
            // ended with a barrier
            ent = cs.ent[tid];
        } else {
            uint32_t start = 0, len = 0;
            if (ci < se) {
                ent = __ldg(G.rowS + ci);
                find_slice(G, ci, ci - X.row0, X, start, len);
            }
            // PF (graphs whose rows do not fit L2): each slice's first lines (all of a short
            // slice: at most 64 entries, three 128-byte lines) are requested now, so that
            // the sweep below finds them in L2
            if (PF && len) {
                prefetch_l2(G.rowC + start);
                prefetch_l2(G.rowC + start + min(len - 1, 32u));
                prefetch_l2(G.rowC + start + min(len - 1, 63u));
            }
            const bool islong = len >= (uint32_t)kLongMin;
            const uint32_t slen = islong ? 0u : len;
            // fields: pieces (bits 32..63), non-empty short slices (16..31), short wedges
            // (0..15; at most 63 per centre, so the chunk's sum stays below 2^15)
            const unsigned long long mine =
                ((unsigned long long)(islong ? (len + kPiece - 1) / kPiece : 0u) << 32) |
                ((unsigned long long)(slen != 0u) << 16) | slen;
            unsigned long long total = 0;
            const unsigned long long ex = block_exclusive_scan_u64(mine, total, cs.wsum);
            cs.start[tid] = start;
            cs.len[tid] = len;
            cs.ent[tid] = ent;
            cs.ppiece[tid] = (uint32_t)(ex >> 32);
            if (slen) {
                const uint32_t c = (uint32_t)(ex >> 16) & 0xffffu, off = (uint32_t)ex & 0xffffu;
                cs.sP[c] = off;
                cs.sbase[c] = start - off;
                cs.smeta[c] = (ent & kSignBit) | (uint32_t)tid;
            }
            cs.acc[tid] = 0;
            if (tid == kChunk - 1) {
                const uint32_t nz = (uint32_t)(total >> 16) & 0xffffu;
                cs.ppiece[kChunk] = (uint32_t)(total >> 32);
                cs.ns = (uint32_t)total & 0xffffu;
                cs.nz = nz;
                cs.sP[nz] = (uint32_t)total & 0xffffu;
            }
            __syncthreads();
        }
        const uint32_t NS = cs.ns, NP = cs.ppiece[kChunk];
        // short slices: each warp takes an equal contiguous range of the chunk's
        // concatenated short wedges and walks it 32 at a time, lane L on position r + L,
        // so a slice's entries are read by consecutive lanes (coalesced). A lane's slice
        // is its window's first slice plus the number of slice ends at or before its
        // position, counted from a bit mask of the ends inside the window.
        if (NS) {
            const int warp = tid >> 5;
            const uint32_t r0 = (uint32_t)(((unsigned long long)NS * warp) / kTileWarps);
            const uint32_t r1 = (uint32_t)(((unsigned long long)NS * (warp + 1)) / kTileWarps);
            if (r0 < r1)
                walk_short<MODE, Acc<CW>, 2>(ctr, rowC, cs.sP, cs.sbase, cs.smeta, (int)cs.nz, r0, r1,
                                          [&](uint32_t tag, Acc<CW> v) { acc_add<CW>(cs, (int)tag, v); });
        }
        // long slices: warp w sweeps pieces w, w + 16, w + 32, ... (pieces are at most
        // kPiece wedges, so the round robin balances like a shared counter without its
        // atomics). A warp finds the slice of its next piece by scanning forward from the
        // slice of its last one, 32 prefix entries per step.
        if (NP) {
            int jw = 0;
            for (uint32_t pc = (uint32_t)(tid >> 5); pc < NP; pc += kTileWarps) {
                for (;;) {
                    const int idx = jw + 1 + lane;
                    const uint32_t val = idx <= kChunk ? cs.ppiece[idx] : 0xffffffffu;
                    const unsigned b = __ballot_sync(kFull, val <= pc);
                    jw += __popc(b);
                    if (b != kFull) break;
                }
                const int j = jw;
                const uint32_t off = (pc - cs.ppiece[j]) * (uint32_t)kPiece;
                const uint32_t n = min((uint32_t)kPiece, cs.len[j] - off);
                const uint32_t s = cs.start[j] + off;
                const uint32_t sk = Ctr::sign_key(cs.ent[j] & kSignBit);
                Acc<CW> acc = 0;
                const uint32_t head = min(n, (4u - (s & 3u)) & 3u);
                if ((uint32_t)lane < head) wedge<MODE, CW>(ctr, __ldg(rowC + s + lane), sk, acc);
                const uint32_t m4 = (n - head) >> 2;
                const uint4 *v4 = reinterpret_cast<const uint4 *>(rowC + s + head);
                // two 16-byte loads in flight per lane (and, in the centre pass, two
                // accumulators so that the additions of the two groups do not chain)
                Acc<CW> acc2 = 0;
                for (uint32_t q = lane; q < m4; q += 64) {
                    const uint4 xa = __ldg(v4 + q);
                    const bool has_b = q + 32 < m4;
                    const uint4 xb = has_b ? __ldg(v4 + q + 32) : make_uint4(0u, 0u, 0u, 0u);
                    wedge<MODE, CW>(ctr, xa.x, sk, acc);
                    wedge<MODE, CW>(ctr, xa.y, sk, acc);
                    wedge<MODE, CW>(ctr, xa.z, sk, acc);
                    wedge<MODE, CW>(ctr, xa.w, sk, acc);
                    if (has_b) {
                        wedge<MODE, CW>(ctr, xb.x, sk, acc2);
                        wedge<MODE, CW>(ctr, xb.y, sk, acc2);
                        wedge<MODE, CW>(ctr, xb.z, sk, acc2);
                        wedge<MODE, CW>(ctr, xb.w, sk, acc2);
                    }
                }
                acc += acc2;
                const uint32_t rest = (n - head) & 3u;
                if ((uint32_t)lane < rest) wedge<MODE, CW>(ctr, __ldg(rowC + s + head + 4 * m4 + lane), sk, acc);
                if (MODE == 1) {
                    // the piece's sum of counts minus one per wedge
                    const Acc<CW> tot = warp_total(acc) - (Acc<CW>)n;
                    if (lane == 0 && tot) acc_add<CW>(cs, j, tot);
                }
            }
        }
        __syncthreads();
        if (MODE == 1 && ci < se) {
            const unsigned long long mine = acc_get<CW>(cs, tid);
            if (X.single)
                centre_carry += mine;   // flushed once per item
            else if (mine)
                red_add(G.bC + (ent & kIdMask), mine);
        }
    }
}

__device__ __forceinline__ void pair_total(unsigned long long p, unsigned long long m,
                                           unsigned long long *bS, uint32_t w,
                                           unsigned long long &bal, unsigned long long &unb) {
    const unsigned long long f = choose2(p) + choose2(m);
    bal += f;
    unb += p * m;
    if (bS && f) red_add(bS + w, f);
}

// Reads, reduces and clears the tile of endpoints [lo, hi), lo being the tile's origin
// (BlockTile::origin: with 8-bit counters an odd first endpoint leaves the word's first
// slot, endpoint lo - 1, unbumped). Words past the last endpoint in the final 16-byte
// group are never bumped and stay zero. With 8-bit
// counters a word holds the bytes (p0, n0, p1, n1) of two endpoints, and
// sum C(x, 2) = (sum x^2 - sum x) / 2 over its bytes, while p0 n0 + p1 n1 is half the
// byte dot product of the word with its pair-swapped self: three dp4a per word.
template <int CW>
__device__ __forceinline__ void tile_epilogue(uint32_t *tile, uint32_t lo, uint32_t hi,
                                              unsigned long long *bS, unsigned long long &bal,
                                              unsigned long long &unb) {
    const uint32_t n = hi - lo;
    const uint32_t words = CW == 0 ? (n + 1) / 2 : (CW == 1 ? n : 2 * n);
    const uint32_t n4 = (words + 3) / 4;
    uint4 *t4 = reinterpret_cast<uint4 *>(tile);
    for (uint32_t i = threadIdx.x; i < n4; i += blockDim.x) {
        const uint4 q = t4[i];
        if ((q.x | q.y | q.z | q.w) == 0) continue;
        t4[i] = make_uint4(0, 0, 0, 0);
        if (CW == 0) {
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
            uint32_t sq = 0, s1 = 0, pn2 = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                sq = __dp4a(w4[k], w4[k], sq);
                s1 = __dp4a(w4[k], 0x01010101u, s1);
                pn2 = __dp4a(w4[k], __byte_perm(w4[k], 0u, 0x2301), pn2);
            }
            bal += (sq - s1) >> 1;
            unb += pn2 >> 1;
            if (bS) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    // a word whose four counts are all at most 1 closes no butterfly
                    if ((w4[k] & 0xfefefefeu) == 0) continue;
                    const uint32_t lo16 = w4[k] & 0xffffu, hi16 = w4[k] >> 16;
                    const uint32_t f0 = (__dp4a(lo16, lo16, 0u) - __dp4a(lo16, 0x0101u, 0u)) >> 1;
                    const uint32_t f1 = (__dp4a(hi16, hi16, 0u) - __dp4a(hi16, 0x0101u, 0u)) >> 1;
                    if (f0) red_add(bS + lo + 8 * i + 2 * k, f0);
                    if (f1) red_add(bS + lo + 8 * i + 2 * k + 1, f1);
                }
            }
        } else if (CW == 1) {
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t p = w4[k] & 0xffffu, m = w4[k] >> 16;
                // each product is even and below 2^32, so the halves add without overflow
                const uint32_t f = ((p * (p - (p > 0))) >> 1) + ((m * (m - (m > 0))) >> 1);
                bal += f;
                unb += p * m;
                if (bS && f) red_add(bS + lo + 4 * i + k, f);
            }
        } else {
            pair_total(q.x, q.y, bS, lo + 2 * i, bal, unb);
            pair_total(q.z, q.w, bS, lo + 2 * i + 1, bal, unb);
        }
    }
}

template <int CW, bool PF>
__device__ void run_tile_item(const DevGraph &G, const TileItem &item, int tile_words, uint32_t *tile,
                              ChunkSmem &cs, unsigned long long &bal, unsigned long long &unb) {
    const int a = item.anchor;
    const int64_t sb = G.rowS_off[a], se = G.rowS_off[a + 1];
    const uint32_t ept = endpoints_per_tile(CW, (uint32_t)tile_words);
    SweepCtx X;
    X.range_lo = G.orient_low ? 0u : (uint32_t)a + 1u;
    X.range_hi = G.orient_low ? (uint32_t)a : (uint32_t)G.nS;
    const int t0 = item.tile_begin, t1 = tile_end_of(item);
    X.nt = (int)((X.range_hi - X.range_lo + ept - 1) / ept);
    X.single = se - sb <= kChunk;
    X.deg = se - sb;
    X.row0 = sb;
    X.bbase = G.boff ? G.boff[a] : 0;
    unsigned long long centre_carry = 0;   // single chunk: this thread's centre, all tiles
    for (int t = t0; t < t1; ++t) {
        X.t = t;
        X.lo = X.range_lo + (uint32_t)t * ept;
        X.hi = min(X.lo + ept, X.range_hi);
        const BlockTile<CW> ctr(tile, X.lo);
        block_sweep<0, CW, BlockTile<CW>, PF>(G, sb, se, X, ctr, cs, centre_carry);
        if (G.bC) block_sweep<1, CW, BlockTile<CW>, PF>(G, sb, se, X, ctr, cs, centre_carry);
        tile_epilogue<CW>(tile, BlockTile<CW>::origin(X.lo), X.hi, G.bS, bal, unb);
        // the next tile's sweep must not bump words the epilogue is still clearing; after
        // the last tile the kernel's item barrier does that
        if (t + 1 < t1) __syncthreads();
    }
    if (centre_carry) red_add(G.bC + (cs.ent[threadIdx.x] & kIdMask), centre_carry);
}

// One tile [X.lo, X.hi) of an anchor: the count sweep, the centre sweep (per-vertex
// counts), the epilogue.
template <int CW, bool PF>
__device__ void tile_pass(const DevGraph &G, int64_t sb, int64_t se, const SweepCtx &X, uint32_t *tile,
                          ChunkSmem &cs, unsigned long long &centre_carry, unsigned long long &bal,
                          unsigned long long &unb, bool last) {
    const BlockTile<CW> ctr(tile, X.lo);
    block_sweep<0, CW, BlockTile<CW>, PF>(G, sb, se, X, ctr, cs, centre_carry);
    if (G.bC) block_sweep<1, CW, BlockTile<CW>, PF>(G, sb, se, X, ctr, cs, centre_carry);
    tile_epilogue<CW>(tile, BlockTile<CW>::origin(X.lo), X.hi, G.bS, bal, unb);
    if (!last) __syncthreads();   // (see run_tile_item)
}

// An item whose tiles choose their counter width one by one (the tile boundaries are the
// same walk that preparation used for the boundary table).
template <bool PF>
__device__ void run_tile_item_var(const DevGraph &G, const TileItem &item, int tile_words, uint32_t *tile,
                                  ChunkSmem &cs, unsigned long long &bal, unsigned long long &unb) {
    const int a = item.anchor;
    const int64_t sb = G.rowS_off[a], se = G.rowS_off[a + 1];
    const unsigned long long deg = (unsigned long long)(se - sb);
    const unsigned long long bound = deg < G.wl[a] ? deg : G.wl[a];
    SweepCtx X;
    X.range_lo = G.orient_low ? 0u : (uint32_t)a + 1u;
    X.range_hi = G.orient_low ? (uint32_t)a : (uint32_t)G.nS;
    const int t0 = item.tile_begin, t1 = tile_end_of(item);
    X.nt = var_tile_count(G.rowS_off, bound, X.range_lo, X.range_hi, (uint32_t)tile_words);
    X.single = se - sb <= kChunk;
    X.deg = se - sb;
    X.row0 = sb;
    X.bbase = G.boff ? G.boff[a] : 0;
    VarTile vt = var_tile_at(G.rowS_off, bound, X.range_lo, X.range_hi, (uint32_t)tile_words);
    for (int t = 0; t < t0; ++t) vt = var_tile_at(G.rowS_off, bound, vt.hi, X.range_hi, (uint32_t)tile_words);
    unsigned long long centre_carry = 0;   // single chunk: this thread's centre, all tiles
    for (int t = t0; t < t1; ++t) {
        X.t = t;
        X.lo = vt.lo;
        X.hi = vt.hi;
        const bool last = t + 1 == t1;
        switch (vt.cw) {
            case 0: tile_pass<0, PF>(G, sb, se, X, tile, cs, centre_carry, bal, unb, last); break;
            case 1: tile_pass<1, PF>(G, sb, se, X, tile, cs, centre_carry, bal, unb, last); break;
            default: tile_pass<2, PF>(G, sb, se, X, tile, cs, centre_carry, bal, unb, last); break;
        }
        if (t + 1 < t1) vt = var_tile_at(G.rowS_off, bound, vt.hi, X.range_hi, (uint32_t)tile_words);
    }
    if (centre_carry) red_add(G.bC + (cs.ent[threadIdx.x] & kIdMask), centre_carry);
}

// ----------------------------------------------------------------------------- centre-split tiles
//
// An anchor with more wedges than its tiles can spread over the blocks (a hub with a
// million centres and a handful of tiles would otherwise run alone for the whole launch)
// has every tile cut into parts by centres. Part k of K sweeps the k-th K-th of the
// anchor's S -> C row into its own shared tile, then adds the tile into the group's
// merged counters in global memory (cs_buf, two 32-bit counters per endpoint). Counting
// pairs needs the complete counts: without per-vertex output the part that arrives last
// (cs_arrive) loads the merged counters back into its tile and runs the usual epilogue;
// with per-vertex output a second launch (k_tile_cs) gives every part the merged tile for
// its centre pass, and the last one of each group runs the epilogue.

__device__ __forceinline__ void red_add_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.global.add.u32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v) : "memory");
}

// Words of a tile whose endpoints run from origin org to hi (the epilogue's count).
template <int CW>
__device__ __forceinline__ uint32_t tile_words_of(uint32_t org, uint32_t hi) {
    const uint32_t n = hi - org;
    return CW == 0 ? (n + 1) / 2 : (CW == 1 ? n : 2 * n);
}

// Adds the tile of endpoints [lo, hi) (origin org) into merged counters buf (counter t of
// endpoint w at 2 (w - lo) + t) and clears the tile. Counter c of the tile belongs to
// endpoint org + c / 2 with type c & 1; with 8-bit counters an odd lo leaves the first
// byte pair (endpoint lo - 1) at zero.
template <int CW>
__device__ void flush_tile(uint32_t *tile, uint32_t org, uint32_t lo, uint32_t hi, uint32_t *buf) {
    const uint32_t words = tile_words_of<CW>(org, hi);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) {
        const uint32_t x = tile[i];
        if (x == 0) continue;
        tile[i] = 0;
        if (CW == 0) {
#pragma unroll
            for (uint32_t b = 0; b < 4; ++b) {
                const uint32_t v = (x >> (8 * b)) & 0xffu, w = org + 2 * i + (b >> 1);
                if (v && w >= lo) red_add_u32(buf + 2 * (w - lo) + (b & 1), v);
            }
        } else if (CW == 1) {
            if (x & 0xffffu) red_add_u32(buf + 2 * i, x & 0xffffu);
            if (x >> 16) red_add_u32(buf + 2 * i + 1, x >> 16);
        } else {
            red_add_u32(buf + i, x);
        }
    }
}

// Writes merged counters buf of endpoints [lo, hi) into a cleared tile (origin org) at
// its width; every count fits, since the width was chosen from a bound on the full count.
template <int CW>
__device__ void load_tile(uint32_t *tile, uint32_t org, uint32_t lo, uint32_t hi, const uint32_t *buf) {
    const uint32_t words = tile_words_of<CW>(org, hi);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) {
        uint32_t x = 0;
        if (CW == 0) {
#pragma unroll
            for (uint32_t b = 0; b < 4; ++b) {
                const uint32_t w = org + 2 * i + (b >> 1);
                if (w >= lo && w < hi) x |= __ldcg(buf + 2 * (w - lo) + (b & 1)) << (8 * b);
            }
        } else if (CW == 1) {
            x = __ldcg(buf + 2 * i) | (__ldcg(buf + 2 * i + 1) << 16);
        } else {
            x = __ldcg(buf + i);
        }
        tile[i] = x;
    }
}

template <int CW>
__device__ __forceinline__ void clear_tile(uint32_t *tile, uint32_t org, uint32_t hi) {
    const uint32_t words = tile_words_of<CW>(org, hi);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) tile[i] = 0;
}

// The tile (X.lo, X.hi, width *cw) and the centre range [*pb, *pe) of centre-split item
// `item`, with its record.
__device__ void cs_setup(const DevGraph &G, const TileItem &item, int tile_words, SweepCtx &X,
                         int64_t &pb, int64_t &pe, int &cw, CentreSplit &d) {
    d = G.cs_desc[item.tile_begin];
    const int a = item.anchor;
    const int64_t sb = G.rowS_off[a], se = G.rowS_off[a + 1];
    X.range_lo = G.orient_low ? 0u : (uint32_t)a + 1u;
    X.range_hi = G.orient_low ? (uint32_t)a : (uint32_t)G.nS;
    X.deg = se - sb;
    X.row0 = sb;
    X.single = false;
    X.bbase = G.boff ? G.boff[a] : 0;
    X.t = d.tile;
    const int w = tile_width_of(item);
    if (w == kWidthPerTile) {
        const unsigned long long deg = (unsigned long long)X.deg;
        const unsigned long long bound = deg < G.wl[a] ? deg : G.wl[a];
        X.nt = var_tile_count(G.rowS_off, bound, X.range_lo, X.range_hi, (uint32_t)tile_words);
        VarTile vt = var_tile_at(G.rowS_off, bound, X.range_lo, X.range_hi, (uint32_t)tile_words);
        for (int t = 0; t < d.tile; ++t) vt = var_tile_at(G.rowS_off, bound, vt.hi, X.range_hi, (uint32_t)tile_words);
        X.lo = vt.lo;
        X.hi = vt.hi;
        cw = vt.cw;
    } else {
        const uint32_t ept = endpoints_per_tile(w, (uint32_t)tile_words);
        X.nt = (int)((X.range_hi - X.range_lo + ept - 1) / ept);
        X.lo = X.range_lo + (uint32_t)d.tile * ept;
        X.hi = min(X.lo + ept, X.range_hi);
        cw = w;
    }
    pb = sb + X.deg * d.part / d.parts;
    pe = sb + X.deg * (d.part + 1) / d.parts;
}

// The count pass of one part (inside the tile kernel). Without per-vertex output the
// last part of the group completes the tile: bal / unb receive its pair totals.
template <int CW, bool PF>
__device__ void cs_count_part(const DevGraph &G, const SweepCtx &X, int64_t pb, int64_t pe,
                              const CentreSplit &d, uint32_t *tile, ChunkSmem &cs, int *s_last,
                              unsigned long long &bal, unsigned long long &unb) {
    const BlockTile<CW> ctr(tile, X.lo);
    unsigned long long carry = 0;
    block_sweep<0, CW, BlockTile<CW>, PF>(G, pb, pe, X, ctr, cs, carry);
    uint32_t *buf = G.cs_buf + (int64_t)d.group * G.cs_group_words;
    const uint32_t org = BlockTile<CW>::origin(X.lo);
    flush_tile<CW>(tile, org, X.lo, X.hi, buf);
    if (G.bC) {
        __syncthreads();
        return;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_last = atomicAdd(G.cs_arrive + d.group, 1u) == (unsigned)(d.parts - 1);
    __syncthreads();
    if (*s_last) {
        __threadfence();
        load_tile<CW>(tile, org, X.lo, X.hi, buf);
        __syncthreads();
        tile_epilogue<CW>(tile, org, X.hi, G.bS, bal, unb);
    }
    __syncthreads();
}

template <bool PF>
__device__ void run_cs_count(const DevGraph &G, const TileItem &item, int tile_words, uint32_t *tile,
                             ChunkSmem &cs, int *s_last, unsigned long long &bal, unsigned long long &unb) {
    SweepCtx X;
    int64_t pb, pe;
    int cw;
    CentreSplit d;
    cs_setup(G, item, tile_words, X, pb, pe, cw, d);
    switch (cw) {
        case 0: cs_count_part<0, PF>(G, X, pb, pe, d, tile, cs, s_last, bal, unb); break;
        case 1: cs_count_part<1, PF>(G, X, pb, pe, d, tile, cs, s_last, bal, unb); break;
        default: cs_count_part<2, PF>(G, X, pb, pe, d, tile, cs, s_last, bal, unb); break;
    }
}

// The centre pass of one part (per-vertex output, after the tile kernel): the merged
// counts go into the tile, the part's slices are swept once more for their centres'
// sums, and the last part of the group runs the epilogue (per-endpoint sums, totals).
template <int CW, bool PF>
__device__ void cs_centre_part(const DevGraph &G, const SweepCtx &X, int64_t pb, int64_t pe,
                               const CentreSplit &d, uint32_t *tile, ChunkSmem &cs, int *s_last,
                               unsigned long long &bal, unsigned long long &unb) {
    const uint32_t org = BlockTile<CW>::origin(X.lo);
    load_tile<CW>(tile, org, X.lo, X.hi, G.cs_buf + (int64_t)d.group * G.cs_group_words);
    __syncthreads();
    const BlockTile<CW> ctr(tile, X.lo);
    unsigned long long carry = 0;
    block_sweep<1, CW, BlockTile<CW>, PF>(G, pb, pe, X, ctr, cs, carry);
    if (threadIdx.x == 0) *s_last = atomicAdd(G.cs_arrive + d.group, 1u) == (unsigned)(d.parts - 1);
    __syncthreads();
    if (*s_last)
        tile_epilogue<CW>(tile, org, X.hi, G.bS, bal, unb);
    else
        clear_tile<CW>(tile, org, X.hi);
    __syncthreads();
}

// Persistent blocks pop (anchor, tile range) items, heaviest first. PF: the graphs' rows
// are much larger than L2 (slices are prefetched into L2 as their chunk is set up).
template <bool PF>
__global__ void __launch_bounds__(kTileThreads, 2)
k_tile(const DevGraph *__restrict__ graphs, const TileItem *__restrict__ items, int n_items,
       unsigned *head, int tile_words, int schedule, long long *item_cycles) {
    const bool static_schedule = schedule == kScheduleStatic;
    extern __shared__ uint4 smem_tile[];
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_tile);
    __shared__ ChunkSmem cs;
    __shared__ int s_item[2], s_last;
    __shared__ unsigned long long s_red[2][kTileWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < tile_words + kTileSlackWords; i += blockDim.x) tile[i] = 0;
    int next_static = blockIdx.x;
    // Thread 0 publishes the next item before the barrier that ends the current one, so
    // that one barrier serves both (the slots alternate, so the write never meets a read
    // of the current item's slot). With kScheduleQueueAhead, past the queue's heavy head
    // it also takes the item after that one item early, so that the atomic's latency
    // hides behind the work; near the head a block holding a second heavy item would end
    // the launch late (and with per-vertex counts, whose items take twice as long, it
    // measured slower throughout).
    auto pop = [&]() -> int {
        if (static_schedule) {
            const int i = next_static;
            next_static += gridDim.x;
            return i;
        }
        return (int)atomicAdd(head, 1u);
    };
    const int deep = schedule == kScheduleQueueAhead ? 8 * (int)gridDim.x : INT_MAX;
    int ahead = -1;
    if (threadIdx.x == 0) s_item[0] = pop();
    auto take = [&](int slot) {
        const int nx = ahead >= 0 ? ahead : pop();
        s_item[slot] = nx;
        ahead = nx >= deep ? pop() : -1;
    };
    __syncthreads();
    for (int slot = 0;; slot ^= 1) {
        const int it = s_item[slot];
        if (it >= n_items) break;
        const TileItem item = items[it];
        const DevGraph &G = graphs[item.graph];
        const long long t_start = item_cycles ? clock64() : 0;
        unsigned long long bal = 0, unb = 0;
        if (is_centre_split(item)) {
            run_cs_count<PF>(G, item, tile_words, tile, cs, &s_last, bal, unb);
        } else {
            switch (tile_width_of(item)) {
                case 0: run_tile_item<0, PF>(G, item, tile_words, tile, cs, bal, unb); break;
                case 1: run_tile_item<1, PF>(G, item, tile_words, tile, cs, bal, unb); break;
                case 2: run_tile_item<2, PF>(G, item, tile_words, tile, cs, bal, unb); break;
                default: run_tile_item_var<PF>(G, item, tile_words, tile, cs, bal, unb); break;
            }
        }
        bal = warp_sum(bal);
        unb = warp_sum(unb);
        if (lane == 0) {
            s_red[0][warp] = bal;
            s_red[1][warp] = unb;
        }
        if (threadIdx.x == 0) take(slot ^ 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long B = 0, U = 0;
            for (int w = 0; w < kTileWarps; ++w) {
                B += s_red[0][w];
                U += s_red[1][w];
            }
            if (B) red_add(G.totals + 0, B);
            if (U) red_add(G.totals + 1, U);
            if (G.bS && B) red_add(G.bS + item.anchor, B);
            // the item's duration on this SM (cost-model labels; off when NULL)
            if (item_cycles) item_cycles[it] = clock64() - t_start;
        }
    }
}

// Per-vertex output: the centre pass of every centre-split item (after the tile kernel
// has merged all parts' counts), persistent blocks over the centre-split list.
template <bool PF>
__global__ void __launch_bounds__(kTileThreads, 2)
k_tile_cs(const DevGraph *__restrict__ graphs, const TileItem *__restrict__ items, int n_items,
          unsigned *head, int tile_words) {
    extern __shared__ uint4 smem_tile[];
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_tile);
    __shared__ ChunkSmem cs;
    __shared__ int s_item, s_last;
    __shared__ unsigned long long s_red[2][kTileWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < tile_words + kTileSlackWords; i += blockDim.x) tile[i] = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const TileItem item = items[it];
        const DevGraph &G = graphs[item.graph];
        SweepCtx X;
        int64_t pb, pe;
        int cw;
        CentreSplit d;
        cs_setup(G, item, tile_words, X, pb, pe, cw, d);
        unsigned long long bal = 0, unb = 0;
        switch (cw) {
            case 0: cs_centre_part<0, PF>(G, X, pb, pe, d, tile, cs, &s_last, bal, unb); break;
            case 1: cs_centre_part<1, PF>(G, X, pb, pe, d, tile, cs, &s_last, bal, unb); break;
            default: cs_centre_part<2, PF>(G, X, pb, pe, d, tile, cs, &s_last, bal, unb); break;
        }
        bal = warp_sum(bal);
        unb = warp_sum(unb);
        if (lane == 0) {
            s_red[0][warp] = bal;
            s_red[1][warp] = unb;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long B = 0, U = 0;
            for (int w = 0; w < kTileWarps; ++w) {
                B += s_red[0][w];
                U += s_red[1][w];
            }
            if (B) red_add(G.totals + 0, B);
            if (U) red_add(G.totals + 1, U);
            if (G.bS && B) red_add(G.bS + item.anchor, B);
        }
    }
}

__global__ void __launch_bounds__(kHashThreads, 5)
k_warp_hash(const DevGraph *__restrict__ graphs, const HashItem *__restrict__ items, int n_items,
            QueueState *q, int chunk, int slots_lg) {
    extern __shared__ uint4 smem_hash[];
    __shared__ uint32_t s_acc[kHashWarps][32];
    __shared__ WarpStage s_stage[kHashWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // each warp's table holds 2^slots_lg slots: twice the largest wedge count of the
    // launch's items, so that small tables leave room for more resident warps
    const int slots = 1 << slots_lg;
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem_hash) + warp * 2 * slots;
    uint32_t *vals = keys + slots;
    for (int i = lane; i < slots; i += 32) {
        keys[i] = kEmpty;
        vals[i] = 0;
    }
    __syncwarp();
    // items come `chunk` at a time from the queue, so that the head's atomics do not
    // serialise a stream of light anchors
    int it = 0, it_end = 0;
    for (;; ++it) {
        if (it >= it_end) {
            if (lane == 0) it = (int)atomicAdd(&q->warp_head, (unsigned)chunk);
            it = __shfl_sync(kFull, it, 0);
            it_end = min(it + chunk, n_items);
        }
        if (it >= n_items) break;
        const HashItem item = items[it];
        const DevGraph &G = graphs[item.graph];
        const int a = item.anchor;
        const int64_t sb = G.rowS_off[a], se = G.rowS_off[a + 1];
        // table of 2^k >= 2 * wedges slots (at least 64)
        int lg = 6;
        while ((1 << lg) < 2 * item.wedges && lg < slots_lg) ++lg;
        const HashCounter ctr{keys, vals, (1u << lg) - 1u, 32 - lg, &q->error};
        warp_sweep<0, 1>(G, sb, se, ctr, nullptr, nullptr, s_stage[warp]);
        __syncwarp();
        if (G.bC) {
            warp_sweep<1, 1>(G, sb, se, ctr, nullptr, s_acc[warp], s_stage[warp]);
            __syncwarp();
        }
        unsigned long long bal = 0, unb = 0;
        for (int i = lane; i <= (int)ctr.mask; i += 32) {
            const uint32_t k = keys[i];
            if (k == kEmpty) continue;
            const uint32_t x = vals[i];
            const unsigned long long p = x & 0xffffu, m = x >> 16;
            const unsigned long long f = choose2(p) + choose2(m);
            bal += f;
            unb += p * m;
            if (G.bS && f) red_add(G.bS + k, f);
            keys[i] = kEmpty;
            vals[i] = 0;
        }
        bal = warp_sum(bal);
        unb = warp_sum(unb);
        if (lane == 0) {
            if (bal) red_add(G.totals + 0, bal);
            if (unb) red_add(G.totals + 1, unb);
            if (G.bS && bal) red_add(G.bS + a, bal);
        }
        __syncwarp();
    }
}


// ----------------------------------------------------------------------------- group tiles

// Barrier over the GW warps of one group (a named barrier per group; a warp sync for a
// group of one warp).
template <int GW>
__device__ __forceinline__ void group_sync(int grp) {
    if (GW == 1)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(GW * 32) : "memory");
}

// A group of GW warps with a dense counter table of GW * kWtWords words counts one anchor
// whose whole endpoint range fits the table (single-tile anchors of small and mid-sized
// graphs): the group's warps share its centre batches, and no block barrier is involved.
// Totals of a warp or group tile's endpoints [0, n) without per-vertex updates, 16 bytes
// per thread at a time, then cleared (the block tile's epilogue arithmetic: three dp4a
// per word of 8-bit counters). Words past the span stay zero: nothing bumps them.
template <int CW>
__device__ __forceinline__ void small_tile_totals(uint32_t *tile, uint32_t n, int t, int nt,
                                                  unsigned long long &bal, unsigned long long &unb) {
    const uint32_t words = CW == 0 ? (n + 1) / 2 : (CW == 1 ? n : 2 * n);
    const uint32_t n4 = (words + 3) / 4;
    uint4 *t4 = reinterpret_cast<uint4 *>(tile);
    for (uint32_t i = t; i < n4; i += nt) {
        const uint4 q = t4[i];
        if ((q.x | q.y | q.z | q.w) == 0) continue;
        t4[i] = make_uint4(0u, 0u, 0u, 0u);
        if (CW == 0) {
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
            uint32_t sq = 0, s1 = 0, pn2 = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                sq = __dp4a(w4[k], w4[k], sq);
                s1 = __dp4a(w4[k], 0x01010101u, s1);
                pn2 = __dp4a(w4[k], __byte_perm(w4[k], 0u, 0x2301), pn2);
            }
            bal += (sq - s1) >> 1;
            unb += pn2 >> 1;
        } else if (CW == 1) {
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t p = w4[k] & 0xffffu, m = w4[k] >> 16;
                bal += ((p * (p - (p > 0))) >> 1) + ((m * (m - (m > 0))) >> 1);
                unb += p * m;
            }
        } else {
            bal += choose2(q.x) + choose2(q.y) + choose2(q.z) + choose2(q.w);
            unb += (unsigned long long)q.x * q.y + (unsigned long long)q.z * q.w;
        }
    }
}

template <int GW, int CW>
__device__ void group_tile_item(const DevGraph &G, int a, uint32_t *tile, int grp, int *batch_ctr,
                                uint32_t *sacc, WarpStage &ws) {
    const int lane = threadIdx.x & 31;
    const int gt = threadIdx.x - grp * GW * 32;
    const int64_t sb = G.rowS_off[a], se = G.rowS_off[a + 1];
    const uint32_t lo0 = G.orient_low ? 0u : (uint32_t)a + 1u;
    const uint32_t hi = G.orient_low ? (uint32_t)a : (uint32_t)G.nS;
    const BlockTile<CW> ctr(tile, lo0);
    const uint32_t lo = BlockTile<CW>::origin(lo0);   // the table's first endpoint slot
    if (gt == 0) *batch_ctr = 0;
    group_sync<GW>(grp);
    // a group shares an anchor's centres in batches small enough for every warp to get
    // some: an anchor of few centres with long rows would otherwise keep one warp busy
    const int64_t per_warp = (se - sb + GW - 1) / GW;
    const int batch = GW == 1 ? 32 : (per_warp < 4 ? 4 : (per_warp > 32 ? 32 : (int)per_warp));
    int *const bc = GW == 1 ? nullptr : batch_ctr;   // a single warp takes its batches in order
    warp_sweep<0>(G, sb, se, ctr, bc, nullptr, ws, batch);
    group_sync<GW>(grp);
    if (G.bC) {
        if (gt == 0) *batch_ctr = 0;
        group_sync<GW>(grp);
        warp_sweep<1>(G, sb, se, ctr, bc, sacc, ws, batch);
        group_sync<GW>(grp);
    }
    const uint32_t n = hi - lo;
    unsigned long long bal = 0, unb = 0;
    if (!G.bS) {
        small_tile_totals<CW>(tile, n, gt, GW * 32, bal, unb);
    } else if (CW == 2) {
        for (uint32_t i = gt; i < n; i += GW * 32) {
            const uint32_t p = tile[2 * i], m = tile[2 * i + 1];
            if ((p | m) == 0) continue;
            tile[2 * i] = 0;
            tile[2 * i + 1] = 0;
            pair_total(p, m, G.bS, lo + i, bal, unb);
        }
    } else {
        const uint32_t words = CW == 0 ? (n + 1) / 2 : n;
        for (uint32_t i = gt; i < words; i += GW * 32) {
            const uint32_t x = tile[i];
            if (x == 0) continue;
            tile[i] = 0;
            if (CW == 0) {
                pair_total(x & 0xffu, (x >> 8) & 0xffu, G.bS, lo + 2 * i, bal, unb);
                pair_total((x >> 16) & 0xffu, x >> 24, G.bS, lo + 2 * i + 1, bal, unb);
            } else {
                pair_total(x & 0xffffu, x >> 16, G.bS, lo + i, bal, unb);
            }
        }
    }
    bal = warp_sum(bal);
    unb = warp_sum(unb);
    if (lane == 0) {
        if (bal) red_add(G.totals + 0, bal);
        if (unb) red_add(G.totals + 1, unb);
        if (G.bS && bal) red_add(G.bS + a, bal);
    }
    group_sync<GW>(grp);
}

template <int GW>
__global__ void __launch_bounds__(kWtThreads, 2)
k_group_tile(const DevGraph *__restrict__ graphs, const HashItem *__restrict__ items, int n_items,
             unsigned *head, int chunk) {
    extern __shared__ uint4 smem_wt[];
    __shared__ uint32_t s_acc[kWtWarps][32];
    __shared__ int s_batch[kWtWarps / GW];
    __shared__ int s_item[kWtWarps / GW];
    __shared__ WarpStage s_stage[kWtWarps];
    const int warp = threadIdx.x >> 5;
    const int grp = warp / GW;
    const int gt = threadIdx.x - grp * GW * 32;
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_wt) + grp * (GW * kWtWords);
    for (int i = gt; i < GW * kWtWords; i += GW * 32) tile[i] = 0;
    // items come `chunk` at a time from the queue (see k_warp_hash); a group of several
    // warps has its first thread take each chunk one chunk early, so that the atomic's
    // latency hides behind the current items (single warps measured slower that way)
    int it = 0, it_end = 0;
    int ahead = 0;
    if (GW > 1 && gt == 0) ahead = (int)atomicAdd(head, (unsigned)chunk);
    for (;; ++it) {
        if (it >= it_end) {
            if (gt == 0) {
                if (GW > 1) {
                    s_item[grp] = ahead;
                    ahead = (int)atomicAdd(head, (unsigned)chunk);
                } else {
                    s_item[grp] = (int)atomicAdd(head, (unsigned)chunk);
                }
            }
            group_sync<GW>(grp);
            it = s_item[grp];
            it_end = min(it + chunk, n_items);
            group_sync<GW>(grp);
        }
        if (it >= n_items) break;
        const HashItem item = items[it];
        const DevGraph &G = graphs[item.graph];
        switch (item.cw) {
            case 0: group_tile_item<GW, 0>(G, item.anchor, tile, grp, &s_batch[grp], s_acc[warp], s_stage[warp]); break;
            case 1: group_tile_item<GW, 1>(G, item.anchor, tile, grp, &s_batch[grp], s_acc[warp], s_stage[warp]); break;
            default: group_tile_item<GW, 2>(G, item.anchor, tile, grp, &s_batch[grp], s_acc[warp], s_stage[warp]); break;
        }
    }
}

// ----------------------------------------------------------------------------- motifs

// C(m, k) for k < 2^31: each step multiplies C(m, i) by (m - i) and divides by i + 1,
// which is exact; the 128-bit product is divided in 32-bit digits. Sets ovf and returns 0
// once the value passes 2^64 - 1.
__device__ unsigned long long choose_k(unsigned long long m, uint32_t k, unsigned &ovf) {
    if (k > m) return 0;
    if (k > m - k) k = (uint32_t)(m - k);
    unsigned long long r = 1;
    for (uint32_t i = 0; i < k; ++i) {
        const unsigned long long f = m - i, d = (unsigned long long)i + 1;
        const unsigned long long hi = __umul64hi(r, f), lo = r * f;
        if (hi >= d) {  // the quotient needs more than 64 bits
            ovf = 1;
            return 0;
        }
        const unsigned long long t1 = (hi << 32) | (lo >> 32);
        const unsigned long long q1 = t1 / d, r1 = t1 % d;
        const unsigned long long t0 = (r1 << 32) | (lo & 0xffffffffull);
        r = (q1 << 32) | (t0 / d);
    }
    return r;
}

__device__ __forceinline__ unsigned long long add_ovf(unsigned long long a, unsigned long long b,
                                                      unsigned &ovf) {
    const unsigned long long s = a + b;
    if (s < a) ovf = 1;
    return s;
}

// Sign classes of the endpoints [0, n) of a class tile (Table 7's six rows), then clears
// the tile. The sums are bounded by the graph's butterfly count, which preparation
// checked to fit 64 bits.
template <int CW>
__device__ void class_epilogue(const ClassCounter<CW> &ctr, uint32_t n, unsigned long long (&acc)[6]) {
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
        uint32_t pp, nn, a;
        ctr.read(e, pp, nn, a);
        if ((pp | nn | a) == 0) continue;
        acc[0] += choose2(pp);
        acc[1] += (unsigned long long)pp * nn;
        acc[2] += choose2(nn);
        acc[3] += choose2(a);
        acc[4] += (unsigned long long)pp * a;
        acc[5] += (unsigned long long)nn * a;
    }
    __syncthreads();
    const uint32_t words = n * ClassCounter<CW>::words_per_endpoint;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) ctr.tile[i] = 0;
}

// Balanced and all (2,k)-bicliques of the endpoints [lo, hi) of a counter tile:
// C(p,k) + C(n,k) and C(p+n,k) per endpoint (Lemma 1 extended to k centres), then clears
// the tile.
template <int CW>
__device__ void biclique_epilogue(const TileCounter<CW> &ctr, uint32_t lo, uint32_t hi, uint32_t k,
                                  unsigned long long (&acc)[6], unsigned &ovf) {
    const uint32_t n = hi - lo;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
        const unsigned long long p = ctr.peek(lo + e, 0), m = ctr.peek(lo + e, 1);
        if (p + m < k) continue;
        const unsigned long long bal = add_ovf(choose_k(p, k, ovf), choose_k(m, k, ovf), ovf);
        acc[0] = add_ovf(acc[0], bal, ovf);
        acc[1] = add_ovf(acc[1], choose_k(p + m, k, ovf), ovf);
    }
    __syncthreads();
    const uint32_t words = CW == 0 ? (n + 1) / 2 : (CW == 1 ? n : 2 * n);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) ctr.tile[i] = 0;
}

// One (anchor, tile range) item of a motif count: the count sweep of the tile kernel
// with the motif's counters, then the motif's epilogue. tile_words is the item lists'
// tile size: class tiles use twice the words per endpoint, so their lists are built
// for half the shared-memory tile.
template <int KIND, int CW>
__device__ void run_motif_item(const DevGraph &G, const TileItem &item, int tile_words, uint32_t *tile,
                               ChunkSmem &cs, uint32_t k, unsigned long long (&acc)[6], unsigned &ovf) {
    const int a = item.anchor;
    const int64_t sb = G.rowS_off[a], se = G.rowS_off[a + 1];
    const uint32_t ept = endpoints_per_tile(CW, (uint32_t)tile_words);
    SweepCtx X;
    X.range_lo = G.orient_low ? 0u : (uint32_t)a + 1u;
    X.range_hi = G.orient_low ? (uint32_t)a : (uint32_t)G.nS;
    const int t0 = item.tile_begin, t1 = tile_end_of(item);
    X.nt = (int)((X.range_hi - X.range_lo + ept - 1) / ept);
    X.single = se - sb <= kChunk;
    X.deg = se - sb;
    X.row0 = sb;
    X.bbase = G.boff ? G.boff[a] : 0;
    unsigned long long carry = 0;  // unused: no centre pass
    for (int t = t0; t < t1; ++t) {
        X.t = t;
        X.lo = X.range_lo + (uint32_t)t * ept;
        X.hi = min(X.lo + ept, X.range_hi);
        if (KIND == 1) {
            const ClassCounter<CW> ctr{tile, X.lo};
            block_sweep<0, CW>(G, sb, se, X, ctr, cs, carry);
            class_epilogue<CW>(ctr, X.hi - X.lo, acc);
        } else {
            const TileCounter<CW> ctr{tile, X.lo};
            block_sweep<0, CW>(G, sb, se, X, ctr, cs, carry);
            biclique_epilogue<CW>(ctr, X.lo, X.hi, k, acc, ovf);
        }
        __syncthreads();
    }
}

// Persistent blocks over the motif item list (kind 1: sign classes into out[0..5];
// kind 2: balanced and all (2,k)-bicliques into out[0..1]); out[7] != 0 reports a sum
// past 2^64 - 1.
template <int KIND>
__global__ void __launch_bounds__(kTileThreads, 2)
k_tile_motif(const DevGraph *__restrict__ graphs, const TileItem *__restrict__ items, int n_items,
             unsigned *head, int list_tile_words, int tile_words, uint32_t k,
             unsigned long long *out) {
    extern __shared__ uint4 smem_tile[];
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_tile);
    __shared__ ChunkSmem cs;
    __shared__ int s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < tile_words; i += blockDim.x) tile[i] = 0;
    unsigned long long acc[6] = {0, 0, 0, 0, 0, 0};
    unsigned ovf = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const TileItem item = items[it];
        const DevGraph &G = graphs[item.graph];
        switch (tile_width_of(item)) {
            case 0: run_motif_item<KIND, 0>(G, item, list_tile_words, tile, cs, k, acc, ovf); break;
            case 1: run_motif_item<KIND, 1>(G, item, list_tile_words, tile, cs, k, acc, ovf); break;
            default: run_motif_item<KIND, 2>(G, item, list_tile_words, tile, cs, k, acc, ovf); break;
        }
        __syncthreads();
    }
    // block sums (through the chunk accumulator, idle now), then one add per sum
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        unsigned long long v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = add_ovf(v, __shfl_xor_sync(kFull, v, o), ovf);
        if (lane == 0) cs.acc[warp * 6 + i] = v;
    }
    const int any_ovf = __syncthreads_or((int)ovf);
    if (threadIdx.x < 6) {
        unsigned o2 = 0;
        unsigned long long v = 0;
        for (int w = 0; w < kTileWarps; ++w) v = add_ovf(v, cs.acc[w * 6 + threadIdx.x], o2);
        if (v) {
            const unsigned long long old = atomicAdd(out + threadIdx.x, v);
            if (old + v < old) o2 = 1;
        }
        if (o2) atomicOr(out + 7, 1ull);
    }
    if (threadIdx.x == 0 && any_ovf) atomicOr(out + 7, 1ull);
}

}  // namespace

bbc_status configure_count_kernels() {
    static thread_local int configured_device = -1;
    int dev = 0;
    BBC_CUDA_TRY(cudaGetDevice(&dev));
    if (configured_device != dev) {
        cudaFuncAttributes fa{};
        int maxopt = 0;
        BBC_CUDA_TRY(cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        for (const void *f : {(const void *)k_tile<false>, (const void *)k_tile<true>,
                              (const void *)k_tile_cs<false>, (const void *)k_tile_cs<true>}) {
            BBC_CUDA_TRY(cudaFuncGetAttributes(&fa, f));
            if ((int)fa.sharedSizeBytes > tile_static_smem_bytes()) {
                set_error("tile kernel static shared memory exceeds its budget");
                return BBC_E_CUDA;
            }
            BBC_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              maxopt - (int)fa.sharedSizeBytes));
        }
        for (const void *f : {(const void *)k_tile_motif<1>, (const void *)k_tile_motif<2>}) {
            cudaFuncAttributes fm{};
            BBC_CUDA_TRY(cudaFuncGetAttributes(&fm, f));
            if ((int)fm.sharedSizeBytes > tile_static_smem_bytes()) {
                set_error("motif kernel static shared memory exceeds its budget");
                return BBC_E_CUDA;
            }
            BBC_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              maxopt - (int)fm.sharedSizeBytes));
        }
        BBC_CUDA_TRY(cudaFuncSetAttribute(k_warp_hash, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kHashWarps * 2 * kHashSlots * 4));
        BBC_CUDA_TRY(cudaFuncSetAttribute(k_group_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kWtWarps * kWtWords * 4));
        BBC_CUDA_TRY(cudaFuncSetAttribute(k_group_tile<kGroupWarps>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kWtWarps * kWtWords * 4));
        BBC_CUDA_TRY(cudaFuncSetAttribute(k_group_tile<2 * kGroupWarps>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kWtWarps * kWtWords * 4));
        configured_device = dev;
    }
    return BBC_OK;
}

// Side streams of the calling host thread on the current device: the smaller count
// kernels fork off the caller's stream and join back into it, so each one starts on the
// SMs that the previous one's draining blocks free (inside stream capture the fork and
// join become graph edges).
struct SideStreams {
    int dev = -1;
    cudaStream_t s[3] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[3] = {};
};

bbc_status side_streams(SideStreams *&out) {
    static thread_local SideStreams ss;
    int dev = 0;
    BBC_CUDA_TRY(cudaGetDevice(&dev));
    if (ss.dev != dev) {
        SideStreams fresh;
        for (int i = 0; i < 3; ++i) {
            BBC_CUDA_TRY(cudaStreamCreateWithFlags(&fresh.s[i], cudaStreamNonBlocking));
            BBC_CUDA_TRY(cudaEventCreateWithFlags(&fresh.join[i], cudaEventDisableTiming));
        }
        BBC_CUDA_TRY(cudaEventCreateWithFlags(&fresh.fork, cudaEventDisableTiming));
        fresh.dev = dev;
        ss = fresh;
    }
    out = &ss;
    return BBC_OK;
}

bbc_status ensure_side_streams() {
    SideStreams *ss = nullptr;
    return side_streams(ss);
}

// Resident blocks per SM of the hash kernel with tables of 2^slots_lg slots per warp
// (the occupancy calculator's answer, kept per device and table size).
int hash_blocks_per_sm(int slots_lg) {
    static thread_local int dev_cached = -1;
    static thread_local int occ[11] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 3;
    if (dev != dev_cached) {
        for (int &o : occ) o = 0;
        dev_cached = dev;
    }
    if (occ[slots_lg] == 0) {
        int nb = 0;
        const size_t smem = (size_t)kHashWarps * 2 * ((size_t)1 << slots_lg) * 4;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_warp_hash, kHashThreads, smem) != cudaSuccess ||
            nb < 1)
            nb = 3;
        occ[slots_lg] = nb;
    }
    return occ[slots_lg];
}

bbc_status launch_count(const CountLaunch &L, cudaStream_t st) {
    BBC_TRY(configure_count_kernels());
    const int sms = device_sm_count();
    const Tuning &T = L.tuning;
    if (L.n_tile_items > 0) {
        const int tok = profile_begin(kProfTile, st);
        note_launch();
        // work-queue schedule: persistent blocks (no more than there are items); plain
        // schedule: one block per item
        const int grid = T.plain ? L.n_tile_items : std::min(L.n_tile_items, sms * T.blocks_per_sm);
        auto kern = L.prefetch ? k_tile<true> : k_tile<false>;
        const int schedule = T.plain ? kScheduleStatic : (L.per_vertex ? kScheduleQueue : kScheduleQueueAhead);
        kern<<<grid, kTileThreads, (size_t)(T.tile_words + kTileSlackWords) * 4, st>>>(
            L.graphs, L.tile_items, L.n_tile_items, &L.queue->tile_head, T.tile_words, schedule,
            L.item_cycles);
        BBC_CUDA_TRY(cudaGetLastError());
        profile_end(tok, st);
    }
    // the smaller kernels: each on its own side stream when more than one kernel runs and
    // no per-kernel profile is being taken (it times kernels one after another)
    const int n_small = (L.n_gt_items > 0) + (L.n_wt_items > 0) + (L.n_warp_items > 0);
    const bool fork = n_small > 0 && (L.n_tile_items > 0 || n_small > 1) && !profiling_active();
    SideStreams *ss = nullptr;
    if (fork) {
        BBC_TRY(side_streams(ss));
        BBC_CUDA_TRY(cudaEventRecord(ss->fork, st));
    }
    if (L.n_cs_items > 0) {
        // the centre pass of the centre-split items, once the tile kernel has merged
        // their counts (same stream)
        const int tok = profile_begin(kProfTileCs, st);
        note_launch();
        auto kern = L.prefetch ? k_tile_cs<true> : k_tile_cs<false>;
        kern<<<std::min(L.n_cs_items, sms * T.blocks_per_sm), kTileThreads,
               (size_t)(T.tile_words + kTileSlackWords) * 4, st>>>(L.graphs, L.cs_items, L.n_cs_items,
                                                                    &L.queue->cs_head, T.tile_words);
        BBC_CUDA_TRY(cudaGetLastError());
        profile_end(tok, st);
    }
    int side = 0;
    cudaStream_t main_st = st;
    auto begin_side = [&]() -> cudaStream_t {
        if (!fork) return main_st;
        cudaStreamWaitEvent(ss->s[side], ss->fork, 0);
        return ss->s[side];
    };
    auto end_side = [&](cudaStream_t s2) -> bbc_status {
        if (!fork) return BBC_OK;
        BBC_CUDA_TRY(cudaEventRecord(ss->join[side], s2));
        BBC_CUDA_TRY(cudaStreamWaitEvent(main_st, ss->join[side], 0));
        ++side;
        return BBC_OK;
    };
    if (L.n_gt_items > 0) {
        cudaStream_t st = begin_side();
        const int tok = profile_begin(kProfGroupTile, st);
        note_launch();
        const int groups = kWtWarps / T.group_warps;
        auto kern = T.group_warps == 2 * kGroupWarps ? k_group_tile<2 * kGroupWarps> : k_group_tile<kGroupWarps>;
        kern<<<std::min((L.n_gt_items + groups - 1) / groups, sms * 2), kWtThreads, kWtWarps * kWtWords * 4, st>>>(
            L.graphs, L.gt_items, L.n_gt_items, &L.queue->gt_head, T.queue_chunk);
        BBC_CUDA_TRY(cudaGetLastError());
        profile_end(tok, st);
        BBC_TRY(end_side(st));
    }
    if (L.n_wt_items > 0) {
        cudaStream_t st = begin_side();
        const int tok = profile_begin(kProfWarpTile, st);
        note_launch();
        k_group_tile<1><<<std::min((L.n_wt_items + kWtWarps - 1) / kWtWarps, sms * 2), kWtThreads,
                          kWtWarps * kWtWords * 4, st>>>(
            L.graphs, L.wt_items, L.n_wt_items, &L.queue->wt_head, T.queue_chunk);
        BBC_CUDA_TRY(cudaGetLastError());
        profile_end(tok, st);
        BBC_TRY(end_side(st));
    }
    if (L.n_warp_items > 0) {
        cudaStream_t st = begin_side();
        const int tok = profile_begin(kProfHash, st);
        note_launch();
        int slots_lg = 6;
        while ((1 << slots_lg) < 2 * T.warp_max_wedges && slots_lg < 10) ++slots_lg;
        const size_t smem = (size_t)kHashWarps * 2 * ((size_t)1 << slots_lg) * 4;
        k_warp_hash<<<std::min((L.n_warp_items + kHashWarps - 1) / kHashWarps, sms * hash_blocks_per_sm(slots_lg)),
                      kHashThreads, smem, st>>>(L.graphs, L.warp_items, L.n_warp_items, L.queue,
                                                T.queue_chunk, slots_lg);
        BBC_CUDA_TRY(cudaGetLastError());
        profile_end(tok, st);
        BBC_TRY(end_side(st));
    }
    return BBC_OK;
}

bbc_status launch_motif(const DevGraph *graph, const TileItem *items, int n_items, unsigned *head,
                        int kind, int k, int tile_words, int blocks, unsigned long long *out,
                        cudaStream_t st) {
    BBC_TRY(configure_count_kernels());
    if (n_items <= 0) return BBC_OK;
    const int tok = profile_begin(kProfMotif, st);
    note_launch();
    const size_t smem = (size_t)tile_words * 4;
    if (kind == 1)
        k_tile_motif<1><<<blocks, kTileThreads, smem, st>>>(graph, items, n_items, head, tile_words / 2,
                                                           tile_words, (uint32_t)k, out);
    else
        k_tile_motif<2><<<blocks, kTileThreads, smem, st>>>(graph, items, n_items, head, tile_words,
                                                           tile_words, (uint32_t)k, out);
    BBC_CUDA_TRY(cudaGetLastError());
    profile_end(tok, st);
    return BBC_OK;
}

bbc_status launch_tile_only(const DevGraph *graphs, const TileItem *items, int n_items,
                            unsigned *head, int tile_words, int blocks, cudaStream_t st) {
    BBC_TRY(configure_count_kernels());
    if (n_items <= 0) return BBC_OK;
    note_launch();
    k_tile<false><<<blocks, kTileThreads, (size_t)(tile_words + kTileSlackWords) * 4, st>>>(graphs, items, n_items, head,
                                                                 tile_words, kScheduleQueue, nullptr);
    BBC_CUDA_TRY(cudaGetLastError());
    return BBC_OK;
}

// An upper bound of the tile kernel's static shared memory (checked against the
// compiled kernel when the kernels are configured).
int tile_static_smem_bytes() { return (int)sizeof(ChunkSmem) + 16 * kTileWarps + 512; }

}  // namespace bbc
