// delta.cu -- exact count changes of a batch of edge updates (dynamic signed graphs).
//
// The paper names dynamic signed bipartite graphs (edges added, removed, or re-signed)
// as future work (Sec. VIII). Here a batch D of updates on a prepared graph G gives
// G', and the call returns B(G') - B(G) and the same for unbalanced butterflies without
// recounting G'. By Lemma 1 the counts are sums over pairs {a, w} of the pair side S of
// f(p, n) = C(p,2) + C(n,2) (and p * n), where p and n count the common neighbours
// reached by symmetric and asymmetric wedges. A pair's (p, n) changes only through an
// edge (a, c) or (w, c) in D, so only pairs with a member in A, the set of S vertices that
// an update touches, can change. For every a in A one block recounts a's pair vector in
// G and in G' (all endpoints w, no orientation), and each pair {a, w} adds
// f(G') - f(G) once: at a when w is outside A or ranks above a.
//
// Steps: ids -> ranks (k_rank_of); updates -> (a, c, old sign from the CSR, new sign)
// with range and sign checks (k_map_updates); stable radix sorts by a and by (c, a);
// duplicate and absent-deletion checks (k_check_updates); the distinct anchors A
// (k_anchor_marks + scan); one block per anchor of A (k_delta_anchor), which adds into
// four global counters per endpoint (short centre rows a warp each, long ones the whole
// block) and then reads and clears the whole counter array.
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
    // per block scratch: 4 counters (old p, old n, new p, new n) per endpoint, zero
    // between anchors
    uint32_t *cnt;
    unsigned *next_anchor;
    unsigned long long *out;   // [0] delta balanced, [1] delta unbalanced (two's complement)
};

__device__ __forceinline__ void touch(uint32_t *cnt, uint32_t w, int slot) {
    atomicAdd(cnt + 4 * (size_t)w + slot, 1u);
}

// One centre c of anchor a: its old row, with every entry's new sign looked up among the
// updates, then the insertions at c. Threads t, t + step, ... of the caller's group share
// the row.
__device__ void delta_centre(const DeltaArgs &A, uint32_t a, uint32_t c, uint32_t oa, uint32_t na,
                             uint32_t *cnt, int t, int step) {
    const int64_t b = A.rowC_off[c], e = A.rowC_off[c + 1];
    const int64_t u0 = lower_key(A.key, A.n_upd, (unsigned long long)c << 32);
    const int64_t u1 = lower_key(A.key, A.n_upd, ((unsigned long long)c + 1) << 32);
    for (int64_t j = b + t; j < e; j += step) {
        const uint32_t x = A.rowC[j];
        const uint32_t w = x & kIdMask;
        if (w == a) continue;
        const uint32_t ow = (x >> 31) ? 2u : 1u;
        uint32_t nw = ow;
        if (u1 > u0) {   // an update at this centre may re-sign or delete (w, c)
            int64_t lo = u0, hi = u1;
            const unsigned long long k = ((unsigned long long)c << 32) | w;
            while (lo < hi) {
                const int64_t m = (lo + hi) >> 1;
                if (A.key[m] < k)
                    lo = m + 1;
                else
                    hi = m;
            }
            if (lo < u1 && A.key[lo] == k) nw = A.knew[lo];
        }
        if (oa && ow) touch(cnt, w, oa == ow ? 0 : 1);
        if (na && nw) touch(cnt, w, na == nw ? 2 : 3);
    }
    if (na)
        for (int64_t q = u0 + t; q < u1; q += step) {
            if (A.kold[q] != kAbsent || A.knew[q] == kAbsent) continue;   // insertions only
            const uint32_t w = (uint32_t)(A.key[q] & 0xffffffffull);
            if (w == a) continue;
            touch(cnt, w, na == A.knew[q] ? 2 : 3);
        }
}

// The new sign code of edge (a, c) given its old one.
__device__ __forceinline__ uint32_t new_code(const DeltaArgs &A, uint32_t a, uint32_t c, uint32_t oa) {
    const unsigned long long k = ((unsigned long long)c << 32) | a;
    const int64_t q = lower_key(A.key, A.n_upd, k);
    return (q < A.n_upd && A.key[q] == k) ? A.knew[q] : oa;
}

constexpr int64_t kLongRow = 1024;   // centre rows this long are swept by the whole block

__global__ void __launch_bounds__(kDeltaThreads) k_delta_anchor(DeltaArgs A) {
    __shared__ int s_item;
    __shared__ long long s_red[2][kDeltaWarps];
    uint32_t *cnt = A.cnt + (size_t)blockIdx.x * 4 * (size_t)A.nS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long db = 0, du = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(A.next_anchor, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= A.n_anchors) break;
        const uint32_t a = A.anchors[it];
        const uint32_t sb = A.seg_begin[it];
        const uint32_t se = it + 1 < A.n_anchors ? A.seg_begin[it + 1] : (uint32_t)A.n_upd;
        const int64_t rb = A.rowS_off[a], re = A.rowS_off[a + 1];
        // short centre rows: a warp each
        for (int64_t i = rb + warp; i < re; i += kDeltaWarps) {
            const uint32_t x = A.rowS[i];
            const uint32_t c = x & kIdMask;
            if (A.rowC_off[c + 1] - A.rowC_off[c] >= kLongRow) continue;
            const uint32_t oa = (x >> 31) ? 2u : 1u;
            delta_centre(A, a, c, oa, new_code(A, a, c, oa), cnt, lane, 32);
        }
        for (uint32_t q = sb + warp; q < se; q += kDeltaWarps) {
            const uint32_t c = A.c_by_a[q];
            if (A.old_by_a[q] == kAbsent && A.new_by_a[q] != kAbsent &&
                A.rowC_off[c + 1] - A.rowC_off[c] < kLongRow)
                delta_centre(A, a, c, kAbsent, A.new_by_a[q], cnt, lane, 32);
        }
        // long centre rows: the whole block each
        for (int64_t i = rb; i < re; ++i) {
            const uint32_t x = A.rowS[i];
            const uint32_t c = x & kIdMask;
            if (A.rowC_off[c + 1] - A.rowC_off[c] < kLongRow) continue;
            const uint32_t oa = (x >> 31) ? 2u : 1u;
            delta_centre(A, a, c, oa, new_code(A, a, c, oa), cnt, threadIdx.x, kDeltaThreads);
        }
        for (uint32_t q = sb; q < se; ++q) {
            const uint32_t c = A.c_by_a[q];
            if (A.old_by_a[q] == kAbsent && A.new_by_a[q] != kAbsent &&
                A.rowC_off[c + 1] - A.rowC_off[c] >= kLongRow)
                delta_centre(A, a, c, kAbsent, A.new_by_a[q], cnt, threadIdx.x, kDeltaThreads);
        }
        __syncthreads();
        // every endpoint's four counters, read 16 bytes at a time, then cleared
        uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
        for (int64_t w = threadIdx.x; w < A.nS; w += kDeltaThreads) {
            const uint4 k4 = c4[w];
            if ((k4.x | k4.y | k4.z | k4.w) == 0) continue;
            c4[w] = make_uint4(0u, 0u, 0u, 0u);
            if (A.in_a[w] && (uint32_t)w < a) continue;   // the pair is counted at w
            const long long po = k4.x, no = k4.y, pn = k4.z, nn = k4.w;
            db += (pn * (pn - 1) / 2 + nn * (nn - 1) / 2) - (po * (po - 1) / 2 + no * (no - 1) / 2);
            du += pn * nn - po * no;
        }
        __syncthreads();
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
    if (threadIdx.x == 0) {
        long long b = 0, u = 0;
        for (int w = 0; w < kDeltaWarps; ++w) {
            b += s_red[0][w];
            u += s_red[1][w];
        }
        if (b) atomicAdd(A.out, (unsigned long long)b);
        if (u) atomicAdd(A.out + 1, (unsigned long long)u);
    }
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
        // per-block scratch: 16 bytes per pair-side vertex, at most ~4 GB in all
        const int64_t per_block = 16 * std::max<int64_t>(nS, 1);
        int64_t blocks = std::min<int64_t>(n_anchors, (int64_t)device_sm_count() * 2);
        blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, ((int64_t)4 << 30) / per_block));
        uint32_t *cnt = nullptr;
        BBC_TRY(B.get(&cnt, (size_t)blocks * 4 * (size_t)std::max<int64_t>(nS, 1)));
        BBC_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)blocks * 16 * (size_t)std::max<int64_t>(nS, 1), st));
        DeltaArgs A{g->rowS_off, g->rowS, g->rowC_off, g->rowC, nS, key, kold, knew, n,
                    c_by_a, old_by_a, new_by_a, anchors, seg, (int32_t)n_anchors, in_a,
                    cnt, next, out};
        note_launch();
        k_delta_anchor<<<(unsigned)blocks, kDeltaThreads, 0, st>>>(A);
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
