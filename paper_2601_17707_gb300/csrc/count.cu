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
//     counter array over a window of endpoint ranks (Fig. 4's tiles). Because each C -> S
//     row is sorted by rank, the wedges of centre c that land in the window are one
//     contiguous slice, found by binary search; a warp sweeps long slices with coalesced
//     loads and shares short ones across its lanes. Counters are packed: one 32-bit word
//     per endpoint holding p in the low and n in the high 16 bits (valid while the
//     anchor's counts stay below 65,536), or a 32-bit pair per endpoint otherwise.
//   * k_warp_hash: light anchors (few wedges) get one warp each and a small open-
//     addressing hash table in shared memory, so their cost follows their wedge count
//     and not the width of their endpoint range.
//
// Per-vertex counts (an extension: the paper defines none) follow from the same
// counters: the pair {a, w} adds f = C(p,2) + C(n,2) to both b(a) and b(w); and a wedge
// a - c - w of type t lies in (count_t(a, w) - 1) balanced butterflies through c, so a
// second sweep over the same slices, after the counters are complete, adds that to b(c).
#include "graph.cuh"

namespace bbc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTileThreads = 512;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kLongSlice = 64;            // slices this long are swept by a whole warp
constexpr int kHashThreads = 256;
constexpr int kHashWarps = kHashThreads / 32;
constexpr int kHashSlots = 1024;          // per warp; holds anchors of <= 512 wedges
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

__device__ __forceinline__ unsigned long long choose2(unsigned long long x) {
    return x * (x - (x > 0)) / 2;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// ----------------------------------------------------------------------------- counters

// Dense tile over endpoint ranks [lo, lo + width).
template <bool WIDE>
struct TileCounter {
    uint32_t *tile;
    uint32_t lo;
    __device__ __forceinline__ void bump(uint32_t w, uint32_t t) const {
        const uint32_t i = w - lo;
        if (WIDE)
            atomicAdd(tile + 2 * i + t, 1u);
        else
            atomicAdd(tile + i, 1u << (t << 4));
    }
    __device__ __forceinline__ uint32_t peek(uint32_t w, uint32_t t) const {
        const uint32_t i = w - lo;
        if (WIDE) return tile[2 * i + t];
        return (tile[i] >> (t << 4)) & 0xffffu;
    }
};

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

// One pass over the oriented wedges of anchor rows [sb, se) whose endpoints lie in
// [lo, hi). MODE 0 bumps the counters; MODE 1 (the per-vertex centre pass) reads them
// and adds (count - 1) per wedge to the centre's b. Warps take batches of 32 centres
// from *batch_ctr; lane j of a batch owns centre j and its slice.
template <int MODE, class Counter>
__device__ __forceinline__ void sweep(const DevGraph &G, int64_t sb, int64_t se, uint32_t lo,
                                      uint32_t hi, const Counter &ctr, int *batch_ctr,
                                      uint32_t *sacc) {
    const int lane = threadIdx.x & 31;
    const int64_t nbatch = (se - sb + 31) >> 5;
    const uint32_t *__restrict__ rowC = G.rowC;
    for (;;) {
        int bi = 0;
        if (lane == 0) bi = atomicAdd(batch_ctr, 1);
        bi = __shfl_sync(kFull, bi, 0);
        if (bi >= nbatch) break;
        const int64_t ci = sb + (int64_t)bi * 32 + lane;
        long long b = 0;
        int len = 0;
        uint32_t sg = 0, c = 0;
        if (ci < se) {
            const uint32_t ent = __ldg(G.rowS + ci);
            c = ent & kIdMask;
            sg = ent & kSignBit;
            const int64_t rb = __ldg(G.rowC_off + c), re = __ldg(G.rowC_off + c + 1);
            const int64_t bb = lo == 0 ? rb : lower_bound_rank(rowC, rb, re, lo);
            const int64_t ee = hi >= (uint32_t)G.nS ? re : lower_bound_rank(rowC, bb, re, hi);
            b = bb;
            len = (int)(ee - bb);
        }
        // Long slices: the whole warp sweeps one slice at a time, coalesced.
        unsigned longm = __ballot_sync(kFull, len >= kLongSlice);
        while (longm) {
            const int j = __ffs(longm) - 1;
            longm &= longm - 1;
            const long long bj = __shfl_sync(kFull, b, j);
            const int lj = __shfl_sync(kFull, len, j);
            const uint32_t sj = __shfl_sync(kFull, sg, j);
            unsigned long long acc = 0;
            for (int k = lane; k < lj; k += 32) {
                const uint32_t x = __ldg(rowC + bj + k);
                const uint32_t t = (x ^ sj) >> 31;
                if (MODE == 0)
                    ctr.bump(x & kIdMask, t);
                else
                    acc += ctr.peek(x & kIdMask, t) - 1u;
            }
            if (MODE == 1) {
                acc = warp_sum(acc);
                if (lane == j && acc) atomicAdd(G.bC + c, acc);
            }
        }
        // Short slices: flattened so that every lane has a wedge each step.
        const int sl = len < kLongSlice ? len : 0;
        int incl = sl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - sl;
        if (MODE == 1) {
            sacc[lane] = 0;
            __syncwarp();
        }
        for (int base = 0; base < total; base += 32) {
            const int k = base + lane;
            int j = 0;  // number of lanes whose inclusive end is <= k
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int vv = __shfl_sync(kFull, incl, j + step - 1);
                if (vv <= k) j += step;
            }
            const long long bj = __shfl_sync(kFull, b, j);
            const int ej = __shfl_sync(kFull, excl, j);
            const uint32_t sj = __shfl_sync(kFull, sg, j);
            if (k < total) {
                const uint32_t x = __ldg(rowC + bj + (k - ej));
                const uint32_t t = (x ^ sj) >> 31;
                if (MODE == 0)
                    ctr.bump(x & kIdMask, t);
                else
                    atomicAdd(sacc + j, ctr.peek(x & kIdMask, t) - 1u);
            }
        }
        if (MODE == 1) {
            __syncwarp();
            if (sl > 0 && sacc[lane]) atomicAdd(G.bC + c, (unsigned long long)sacc[lane]);
            __syncwarp();
        }
    }
}

// Reads, reduces and clears the tile of endpoints [lo, hi).
template <bool WIDE>
__device__ __forceinline__ void tile_epilogue(uint32_t *tile, uint32_t lo, uint32_t hi,
                                              unsigned long long *bS, unsigned long long &bal,
                                              unsigned long long &unb) {
    const int n = (int)(hi - lo);
    if (!WIDE) {
        uint4 *t4 = reinterpret_cast<uint4 *>(tile);
        const int n4 = (n + 3) >> 2;  // the tail words beyond n are always zero
        for (int i = threadIdx.x; i < n4; i += blockDim.x) {
            const uint4 q = t4[i];
            if ((q.x | q.y | q.z | q.w) == 0) continue;
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned long long p = w4[k] & 0xffffu, m = w4[k] >> 16;
                const unsigned long long f = choose2(p) + choose2(m);
                bal += f;
                unb += p * m;
                if (bS && f) atomicAdd(bS + lo + 4 * i + k, f);
            }
            t4[i] = make_uint4(0, 0, 0, 0);
        }
    } else {
        uint4 *t4 = reinterpret_cast<uint4 *>(tile);
        const int n2 = (n + 1) >> 1;  // two endpoints per 16 bytes
        for (int i = threadIdx.x; i < n2; i += blockDim.x) {
            const uint4 q = t4[i];
            if ((q.x | q.y | q.z | q.w) == 0) continue;
            const unsigned long long p0 = q.x, m0 = q.y, p1 = q.z, m1 = q.w;
            const unsigned long long f0 = choose2(p0) + choose2(m0);
            const unsigned long long f1 = choose2(p1) + choose2(m1);
            bal += f0 + f1;
            unb += p0 * m0 + p1 * m1;
            if (bS) {
                if (f0) atomicAdd(bS + lo + 2 * i, f0);
                if (f1) atomicAdd(bS + lo + 2 * i + 1, f1);
            }
            t4[i] = make_uint4(0, 0, 0, 0);
        }
    }
}

// ----------------------------------------------------------------------------- kernels

template <bool WIDE>
__global__ void __launch_bounds__(kTileThreads, 2)
k_tile(const DevGraph *__restrict__ graphs, const TileItem *__restrict__ items, int n_items,
       unsigned *head, int tile_words) {
    extern __shared__ uint4 smem_tile[];
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_tile);
    __shared__ int s_item;
    __shared__ int s_batch[2];
    __shared__ uint32_t s_acc[kTileWarps][32];
    __shared__ unsigned long long s_red[2][kTileWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < tile_words; i += blockDim.x) tile[i] = 0;
    const uint32_t ept = WIDE ? (uint32_t)tile_words / 2 : (uint32_t)tile_words;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const TileItem item = items[it];
        const DevGraph &G = graphs[item.graph];
        const int a = item.anchor;
        const int64_t sb = G.rowS_off[a], se = G.rowS_off[a + 1];
        const uint32_t range_lo = G.orient_low ? 0u : (uint32_t)a + 1u;
        const uint32_t range_hi = G.orient_low ? (uint32_t)a : (uint32_t)G.nS;
        unsigned long long bal = 0, unb = 0;
        for (int t = item.tile_begin; t < item.tile_end; ++t) {
            const uint32_t lo = range_lo + (uint32_t)t * ept;
            const uint32_t hi = min(lo + ept, range_hi);
            if (threadIdx.x == 0) {
                s_batch[0] = 0;
                s_batch[1] = 0;
            }
            __syncthreads();
            const TileCounter<WIDE> ctr{tile, lo};
            sweep<0>(G, sb, se, lo, hi, ctr, &s_batch[0], nullptr);
            __syncthreads();
            if (G.bC) {
                sweep<1>(G, sb, se, lo, hi, ctr, &s_batch[1], s_acc[warp]);
                __syncthreads();
            }
            tile_epilogue<WIDE>(tile, lo, hi, G.bS, bal, unb);
            __syncthreads();
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
            if (B) atomicAdd(G.totals + 0, B);
            if (U) atomicAdd(G.totals + 1, U);
            if (G.bS && B) atomicAdd(G.bS + a, B);
        }
    }
}

__global__ void __launch_bounds__(kHashThreads)
k_warp_hash(const DevGraph *__restrict__ graphs, const HashItem *__restrict__ items, int n_items,
            QueueState *q) {
    extern __shared__ uint4 smem_hash[];
    __shared__ uint32_t s_acc[kHashWarps][32];
    __shared__ int s_batch[kHashWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem_hash) + warp * 2 * kHashSlots;
    uint32_t *vals = keys + kHashSlots;
    for (int i = lane; i < kHashSlots; i += 32) {
        keys[i] = kEmpty;
        vals[i] = 0;
    }
    __syncwarp();
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(&q->warp_head, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const HashItem item = items[it];
        const DevGraph &G = graphs[item.graph];
        const int a = item.anchor;
        const int64_t sb = G.rowS_off[a], se = G.rowS_off[a + 1];
        const uint32_t lo = G.orient_low ? 0u : (uint32_t)a + 1u;
        const uint32_t hi = G.orient_low ? (uint32_t)a : (uint32_t)G.nS;
        // table of 2^k >= 2 * wedges slots (at least 64)
        int lg = 6;
        while ((1 << lg) < 2 * item.wedges && lg < 10) ++lg;
        const HashCounter ctr{keys, vals, (1u << lg) - 1u, 32 - lg, &q->error};
        if (lane == 0) s_batch[warp] = 0;
        __syncwarp();
        sweep<0>(G, sb, se, lo, hi, ctr, &s_batch[warp], nullptr);
        __syncwarp();
        if (G.bC) {
            if (lane == 0) s_batch[warp] = 0;
            __syncwarp();
            sweep<1>(G, sb, se, lo, hi, ctr, &s_batch[warp], s_acc[warp]);
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
            if (G.bS && f) atomicAdd(G.bS + k, f);
            keys[i] = kEmpty;
            vals[i] = 0;
        }
        bal = warp_sum(bal);
        unb = warp_sum(unb);
        if (lane == 0) {
            if (bal) atomicAdd(G.totals + 0, bal);
            if (unb) atomicAdd(G.totals + 1, unb);
            if (G.bS && bal) atomicAdd(G.bS + a, bal);
        }
        __syncwarp();
    }
}

}  // namespace

int tile_kernel_smem_bytes(int tile_words, bool) { return tile_words * 4; }

bbc_status configure_count_kernels() {
    static thread_local int configured_device = -1;
    int dev = 0;
    BBC_CUDA_TRY(cudaGetDevice(&dev));
    if (configured_device != dev) {
        int maxopt = 0;
        BBC_CUDA_TRY(cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        BBC_CUDA_TRY(cudaFuncSetAttribute(k_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          maxopt - 4096));
        BBC_CUDA_TRY(cudaFuncSetAttribute(k_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          maxopt - 4096));
        BBC_CUDA_TRY(cudaFuncSetAttribute(k_warp_hash, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kHashWarps * 2 * kHashSlots * 4));
        configured_device = dev;
    }
    return BBC_OK;
}

bbc_status launch_count(const CountLaunch &L, cudaStream_t st) {
    BBC_TRY(configure_count_kernels());
    const int sms = device_sm_count();
    const Tuning &T = L.tuning;
    const size_t tile_smem = (size_t)T.tile_words * 4;
    if (L.n_tile_items > 0) {
        const int grid = sms * T.blocks_per_sm;
        k_tile<false><<<grid, kTileThreads, tile_smem, st>>>(L.graphs, L.tile_items, L.n_tile_items,
                                                             &L.queue->tile_head, T.tile_words);
        BBC_CUDA_TRY(cudaGetLastError());
    }
    if (L.n_wide_items > 0) {
        const int grid = sms * T.blocks_per_sm;
        k_tile<true><<<grid, kTileThreads, tile_smem, st>>>(L.graphs, L.wide_items, L.n_wide_items,
                                                            &L.queue->wide_head, T.tile_words);
        BBC_CUDA_TRY(cudaGetLastError());
    }
    if (L.n_warp_items > 0) {
        const int grid = sms * 3;
        k_warp_hash<<<grid, kHashThreads, kHashWarps * 2 * kHashSlots * 4, st>>>(
            L.graphs, L.warp_items, L.n_warp_items, L.queue);
        BBC_CUDA_TRY(cudaGetLastError());
    }
    return BBC_OK;
}

}  // namespace bbc
