// sort_scan.cu -- the two data-movement primitives of graph preparation: a stable
// least-significant-digit radix sort of (key, value) pairs and a device-wide
// exclusive scan. Both are plain streaming kernels (HBM-bound); tiles are sized so a
// grid spans many multiples of the SM count.
#include "bbc_internal.cuh"

namespace bbc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ----------------------------------------------------------------------------- radix sort

constexpr int kRsWarps = 8;
constexpr int kRsThreads = kRsWarps * 32;
constexpr int kRsRounds = 8;                       // items per lane
constexpr int kRsTile = kRsThreads * kRsRounds;   // 2048 items per block
constexpr int kRsBits = 8;
constexpr int kRsBuckets = 1 << kRsBits;

// Per-tile digit histogram, stored digit-major (hist[d * ntiles + tile]) so that one
// exclusive scan of the whole array yields every tile's output offset per digit.
__global__ void __launch_bounds__(kRsThreads)
k_rs_histogram(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t mask,
               uint32_t *__restrict__ hist, int ntiles) {
    __shared__ uint32_t cnt[kRsBuckets];
    for (int i = threadIdx.x; i < kRsBuckets; i += kRsThreads) cnt[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t idx = base + r * kRsThreads + threadIdx.x;
        const bool valid = idx < n;
        const uint32_t d = valid ? ((__ldg(keys + idx) >> shift) & mask) : (0x100u + lane);
        const unsigned peers = __match_any_sync(kFull, d);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&cnt[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRsBuckets; i += kRsThreads)
        hist[(int64_t)i * ntiles + blockIdx.x] = cnt[i];
}

// Stable scatter. Warp w of a tile owns items [w*256, (w+1)*256) of the tile and walks
// them in 8 rounds of 32 consecutive items; __match_any_sync ranks equal digits within
// a round, a per-warp counter carries ranks across rounds, and a per-digit prefix over
// the warps orders the warps. Together with the scanned histogram this reproduces the
// input order among equal digits.
__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
             uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
             uint32_t mask, const uint32_t *__restrict__ offs, int ntiles) {
    __shared__ uint32_t wcnt[kRsWarps][kRsBuckets];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kRsWarps * kRsBuckets; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)warp * (32 * kRsRounds);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t k[kRsRounds], v[kRsRounds], d[kRsRounds], rk[kRsRounds];
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t idx = base + r * 32 + lane;
        const bool valid = idx < n;
        k[r] = valid ? __ldg(kin + idx) : 0u;
        v[r] = valid ? __ldg(vin + idx) : 0u;
        d[r] = valid ? ((k[r] >> shift) & mask) : (0x100u + lane);
        const unsigned peers = __match_any_sync(kFull, d[r]);
        const uint32_t before = valid ? wcnt[warp][d[r]] : 0u;
        __syncwarp();
        rk[r] = before + (uint32_t)__popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d[r]] = before + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kRsBuckets; dd += kRsThreads) {
        uint32_t run = offs[(int64_t)dd * ntiles + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t c = wcnt[w][dd];
            wcnt[w][dd] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t idx = base + r * 32 + lane;
        if (idx < n) {
            const uint32_t pos = wcnt[warp][d[r]] + rk[r];
            kout[pos] = k[r];
            vout[pos] = v[r];
        }
    }
}

// ----------------------------------------------------------------------------- scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Block-exclusive scan of one value per thread; returns the block total in *total.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T x, T *total) {
    __shared__ T wsum[kScanThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T inc = warp_inclusive_scan(x);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kScanThreads / 32 ? wsum[lane] : T(0);
        const T wi = warp_inclusive_scan(w);
        if (lane < kScanThreads / 32) wsum[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    const T r = wsum[warp] + inc - x;
    __syncthreads();
    return r;
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads)
k_scan_block_sums(const Tin *__restrict__ in, int64_t n, Tout *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    Tout s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        const int64_t idx = base + i;
        if (idx < n) s += (Tout)in[idx];
    }
    __shared__ Tout total;
    block_exclusive_scan<Tout>(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const Tin *__restrict__ in, int64_t n, const Tout *__restrict__ block_prefix,
             Tout *__restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    Tout vals[kScanItems];
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + i;
        vals[i] = idx < n ? (Tout)in[idx] : Tout(0);
        s += vals[i];
    }
    __shared__ Tout total;
    Tout run = block_exclusive_scan<Tout>(s, &total) +
               (block_prefix ? block_prefix[blockIdx.x] : Tout(0));
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += vals[i];
    }
    // The last thread of the last block ends at the grand total; it also fills out[n].
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = run;
}

// Exclusive scan with out[n] = total. Recurses on the per-block sums.
template <class Tin, class Tout>
bbc_status exclusive_scan(const Tin *in, Tout *out, int64_t n, cudaStream_t st) {
    if (n <= 0) {
        BBC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(Tout), st));
        return BBC_OK;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        note_launch();
        k_scan_apply<Tin, Tout><<<1, kScanThreads, 0, st>>>(in, n, nullptr, out);
        BBC_CUDA_TRY(cudaGetLastError());
        return BBC_OK;
    }
    Tout *sums = nullptr, *pref = nullptr;
    BBC_TRY(dev_alloc_n(&sums, (size_t)nb, st));
    bbc_status s = dev_alloc_n(&pref, (size_t)nb + 1, st);
    if (s != BBC_OK) {
        dev_free(sums, st);
        return s;
    }
    note_launch();
    k_scan_block_sums<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums);
    s = exclusive_scan<Tout, Tout>(sums, pref, nb, st);
    if (s == BBC_OK) {
        note_launch();
        k_scan_apply<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, pref, out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(e, "k_scan_apply");
    }
    dev_free(sums, st);
    dev_free(pref, st);
    return s;
}

}  // namespace

bbc_status exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    return exclusive_scan<int32_t, int64_t>(in, out, n, st);
}

bbc_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    return exclusive_scan<int64_t, int64_t>(in, out, n, st);
}

bbc_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t st) {
    return exclusive_scan<uint32_t, uint32_t>(in, out, n, st);
}

bbc_status radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t st) {
    if (n <= 1 || bits <= 0) return BBC_OK;
    if (n >= (int64_t)0xffffffffLL) {
        set_error("radix sort: more than 2^32 - 1 items");
        return BBC_E_INVALID_ARG;
    }
    const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    const int64_t hn = ntiles * kRsBuckets;
    uint32_t *k2 = nullptr, *v2 = nullptr, *hist = nullptr, *offs = nullptr;
    bbc_status s = dev_alloc_n(&k2, (size_t)n, st);
    if (s == BBC_OK) s = dev_alloc_n(&v2, (size_t)n, st);
    if (s == BBC_OK) s = dev_alloc_n(&hist, (size_t)hn, st);
    if (s == BBC_OK) s = dev_alloc_n(&offs, (size_t)hn + 1, st);
    uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
    for (int shift = 0; s == BBC_OK && shift < bits; shift += kRsBits) {
        const int width = bits - shift < kRsBits ? bits - shift : kRsBits;
        const uint32_t mask = (1u << width) - 1u;
        note_launch();
        k_rs_histogram<<<(unsigned)ntiles, kRsThreads, 0, st>>>(ka, n, shift, mask, hist, (int)ntiles);
        s = exclusive_scan_u32(hist, offs, hn, st);
        if (s != BBC_OK) break;
        note_launch();
        k_rs_scatter<<<(unsigned)ntiles, kRsThreads, 0, st>>>(ka, va, kb, vb, n, shift, mask, offs,
                                                               (int)ntiles);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            s = cuda_fail(e, "k_rs_scatter");
            break;
        }
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (s == BBC_OK && ka != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, ka, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) s = cuda_fail(e, "radix sort copy-back");
    }
    dev_free(k2, st);
    dev_free(v2, st);
    dev_free(hist, st);
    dev_free(offs, st);
    return s;
}

}  // namespace bbc
