// costmodel.cu -- a learned cost model for the tile kernel's work items.
//
// The queue of the tile kernel hands out (anchor, tile range) items heaviest first
// (Algorithm 4 orders by a fanout estimate; preparation orders by each item's share of
// its anchor's oriented wedges). An item's real cost also depends on the anchor's degree
// (one slice setup per centre and tile), on the endpoint span it clears, and on where its
// tiles sit in the anchor's range. This file learns that cost from measured item
// durations and reorders the queue by the prediction:
//   * features: eight numbers per tile item, computed on the device from the graph
//     (k_item_features);
//   * labels: the item's duration in SM cycles from an instrumented tile-kernel run,
//     as standardised log cycles (k_labels);
//   * network: 8 -> 32 -> 32 -> 1, ReLU, fp32. One warp evaluates one sample at a time,
//     lane j being hidden unit j in both layers, so forward and backward are register
//     and shuffle work (k_mlp_predict, k_mlp_grad); loss = mean squared error; Adam
//     updates (k_adam);
//   * use: items sorted by predicted cost, heaviest first (bbc_cost_model_order).
// None of this touches the counting arithmetic: any item order gives the same counts.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "graph.cuh"

struct bbc_cost_model {
    int device = 0;
    float *params = nullptr;  // device, kParams
    float *grad = nullptr;    // device, kParams (+1: the loss)
    float *m = nullptr;       // device, Adam first moments
    float *v = nullptr;       // device, Adam second moments
    int step = 0;
    float label_mu = 0.f, label_sd = 1.f;
};

namespace bbc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kF = 8;   // features per item
constexpr int kH = 32;  // hidden units per layer (one per lane)
// parameter layout: W1[kH][kF], b1[kH], W2[kH][kH] (row j = unit j of layer 2), b2[kH],
// w3[kH], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH * kF;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;
constexpr int kParams = kOffB3 + 1;
constexpr int kWarpsPerBlock = 8;

inline unsigned grid_blocks(int64_t n_warps_wanted) {
    int64_t b = (n_warps_wanted + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Features of tile item i (all of order one):
//   0 log1p(anchor wedges) / 16      1 log1p(anchor degree) / 16
//   2 log1p(tiles in the item) / 8   3 log1p(endpoint span of the item) / 16
//   4 first tile / the anchor's tiles 5 counter width / 2
//   6 log1p(|S|) / 16                7 log1p(wedges * item tiles / anchor tiles
//                                      [/ parts of a centre-split tile]) / 16
__global__ void k_item_features(const DevGraph *__restrict__ graphs, const TileItem *__restrict__ items,
                                int n, int tile_words, float *__restrict__ X) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const TileItem it = items[i];
        const DevGraph &G = graphs[it.graph];
        const int a = it.anchor;
        const int cw = tile_width_of(it);
        const double deg = (double)(G.rowS_off[a + 1] - G.rowS_off[a]);
        const double wl = (double)G.wl[a];
        const double ept = cw == 0 ? 2.0 * tile_words : (cw == 1 ? (double)tile_words : tile_words / 2.0);
        const double range = G.orient_low ? (double)a : (double)(G.nS - 1 - a);
        const double nt = fmax(1.0, ceil(range / ept));
        // a centre-split item: one tile, and a 1 / parts share of its centres
        double share = 1.0;
        int t0 = it.tile_begin, t1 = tile_end_of(it);
        if (is_centre_split(it)) {
            const CentreSplit d = G.cs_desc[it.tile_begin];
            t0 = d.tile;
            t1 = d.tile + 1;
            share = 1.0 / d.parts;
        }
        const double span = fmax(0.0, fmin(t1 * ept, range) - t0 * ept);
        float *x = X + (int64_t)i * kF;
        x[0] = (float)(log1p(wl) / 16.0);
        x[1] = (float)(log1p(deg) / 16.0);
        x[2] = (float)(log1p((double)(t1 - t0)) / 8.0);
        x[3] = (float)(log1p(span) / 16.0);
        x[4] = (float)(t0 / nt);
        x[5] = (float)(cw / 2.0);
        x[6] = (float)(log1p((double)G.nS) / 16.0);
        x[7] = (float)(log1p(wl * (t1 - t0) / nt * share) / 16.0);
    }
}

// This lane's weights: W1 row, b1, W2 row, b2, w3 (lane = hidden unit j).
struct LaneWeights {
    float w1[kF], b1, w2[kH], b2, w3, b3;
};

__device__ __forceinline__ void load_weights(const float *__restrict__ P, int lane, LaneWeights &W) {
#pragma unroll
    for (int f = 0; f < kF; ++f) W.w1[f] = P[kOffW1 + lane * kF + f];
    W.b1 = P[kOffB1 + lane];
#pragma unroll
    for (int k = 0; k < kH; ++k) W.w2[k] = P[kOffW2 + lane * kH + k];
    W.b2 = P[kOffB2 + lane];
    W.w3 = P[kOffW3 + lane];
    W.b3 = P[kOffB3];
}

// Forward pass of one sample by a whole warp: lane j ends with z1[j], z2[j] (the
// pre-activations) and the output y (all lanes).
__device__ __forceinline__ float forward(const LaneWeights &W, const float *__restrict__ x, int lane,
                                         float &z1, float &h1, float &z2, float &h2) {
    z1 = W.b1;
#pragma unroll
    for (int f = 0; f < kF; ++f) z1 = fmaf(W.w1[f], x[f], z1);
    h1 = fmaxf(z1, 0.f);
    z2 = W.b2;
#pragma unroll
    for (int k = 0; k < kH; ++k) z2 = fmaf(W.w2[k], __shfl_sync(kFull, h1, k), z2);
    h2 = fmaxf(z2, 0.f);
    float y = W.w3 * h2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(kFull, y, o);
    return y + W.b3;
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_mlp_predict(const float *__restrict__ P, const float *__restrict__ X, int n, float *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int n_warps = gridDim.x * kWarpsPerBlock;
    LaneWeights W;
    load_weights(P, lane, W);
    for (int i = warp; i < n; i += n_warps) {
        float z1, h1, z2, h2;
        const float out = forward(W, X + (int64_t)i * kF, lane, z1, h1, z2, h2);
        if (lane == 0) y[i] = out;
    }
}

// Gradient of L = (1/n) sum_i (y_i - t_i)^2 by backpropagation, accumulated per lane
// over the warp's samples and then added into grad[0..kParams); grad[kParams] += L.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_mlp_grad(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ T, int n,
           float *__restrict__ grad) {
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int n_warps = gridDim.x * kWarpsPerBlock;
    LaneWeights W;
    load_weights(P, lane, W);
    float gw1[kF], gb1 = 0.f, gw2[kH], gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, loss = 0.f;
#pragma unroll
    for (int f = 0; f < kF; ++f) gw1[f] = 0.f;
#pragma unroll
    for (int k = 0; k < kH; ++k) gw2[k] = 0.f;
    const float inv_n = 1.f / (float)n;
    for (int i = warp; i < n; i += n_warps) {
        const float *x = X + (int64_t)i * kF;
        float z1, h1, z2, h2;
        const float y = forward(W, x, lane, z1, h1, z2, h2);
        const float r = y - T[i];
        loss += r * r * inv_n;
        const float dy = 2.f * r * inv_n;   // dL/dy
        gb3 += dy;
        gw3 = fmaf(dy, h2, gw3);
        const float dz2 = z2 > 0.f ? dy * W.w3 : 0.f;   // this lane's unit of layer 2
        gb2 += dz2;
        // dL/dW2[j][k] = dz2[j] h1[k]; dL/dh1[k] = sum_j dz2[j] W2[j][k] (lane k collects)
        float dh1 = 0.f;
#pragma unroll
        for (int k = 0; k < kH; ++k) {
            gw2[k] = fmaf(dz2, __shfl_sync(kFull, h1, k), gw2[k]);
            const float contrib = dz2 * W.w2[k];   // unit j's share of dL/dh1[k]
            float s = contrib;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            if (lane == k) dh1 = s;
        }
        const float dz1 = z1 > 0.f ? dh1 : 0.f;
        gb1 += dz1;
#pragma unroll
        for (int f = 0; f < kF; ++f) gw1[f] = fmaf(dz1, x[f], gw1[f]);
    }
#pragma unroll
    for (int f = 0; f < kF; ++f) atomicAdd(grad + kOffW1 + lane * kF + f, gw1[f]);
    atomicAdd(grad + kOffB1 + lane, gb1);
#pragma unroll
    for (int k = 0; k < kH; ++k) atomicAdd(grad + kOffW2 + lane * kH + k, gw2[k]);
    atomicAdd(grad + kOffB2 + lane, gb2);
    atomicAdd(grad + kOffW3 + lane, gw3);
    if (lane == 0) {
        atomicAdd(grad + kOffB3, gb3);
        atomicAdd(grad + kParams, loss);
    }
}

// Adam (Kingma and Ba 2015) with bias correction.
__global__ void k_adam(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                       float *__restrict__ V, int n, float lr, float beta1, float beta2, float eps,
                       float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = beta1 * M[i] + (1.f - beta1) * g;
        const float v = beta2 * V[i] + (1.f - beta2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// sums[0] += log(c), sums[1] += log(c)^2 over positive cycles
__global__ void k_label_moments(const long long *__restrict__ cyc, int n, double *__restrict__ sums) {
    double s = 0, q = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double l = log((double)(cyc[i] > 0 ? cyc[i] : 1));
        s += l;
        q += l * l;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(kFull, s, o);
        q += __shfl_xor_sync(kFull, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums, s);
        atomicAdd(sums + 1, q);
    }
}

__global__ void k_labels(const long long *__restrict__ cyc, int n, float mu, float sd, float *__restrict__ t) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = (float)((log((double)(cyc[i] > 0 ? cyc[i] : 1)) - mu) / sd);
}

// Descending order of predictions as ascending 32-bit keys.
__global__ void k_order_keys(const float *__restrict__ y, int n, uint32_t *__restrict__ keys,
                             uint32_t *__restrict__ idx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = __float_as_uint(y[i]);
        const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // monotone in y
        keys[i] = ~asc;
        idx[i] = (uint32_t)i;
    }
}

__global__ void k_gather_tile_items(const TileItem *__restrict__ in, const uint32_t *__restrict__ order,
                                    int n, TileItem *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[order[i]];
}

// Device buffers released together when the owner leaves scope.
struct Buffers {
    cudaStream_t st;
    void *p[8];
    int n = 0;
    explicit Buffers(cudaStream_t s) : st(s) {}
    template <class T>
    bbc_status get(T **out, size_t count) {
        const bbc_status s = dev_alloc_n(out, count, st);
        if (s == BBC_OK) p[n++] = *out;
        return s;
    }
    ~Buffers() {
        for (int i = 0; i < n; ++i) dev_free(p[i], st);
    }
};

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

bbc_status model_ready(const bbc_cost_model *m) {
    if (!m || !m->params) {
        set_error("cost model: NULL model");
        return BBC_E_INVALID_ARG;
    }
    return BBC_OK;
}

// Features of g's current tile items into X (device, capacity rows of kF floats).
bbc_status item_features(bbc_graph *g, float *X, int capacity, int *n_items, cudaStream_t st) {
    *n_items = g->n_tile;
    if (g->n_tile > capacity) {
        set_error("item features: capacity below the number of tile items");
        return BBC_E_INVALID_ARG;
    }
    if (g->n_tile == 0) return BBC_OK;
    DevGraph d = host_descriptor(g, false, true);
    BBC_CUDA_TRY(cudaMemcpyAsync(g->dgraph, &d, sizeof d, cudaMemcpyHostToDevice, st));
    note_launch();
    k_item_features<<<(g->n_tile + 255) / 256, 256, 0, st>>>(g->dgraph, g->tile_items, g->n_tile,
                                                             g->items_tuning.tile_words, X);
    BBC_CUDA_TRY(cudaGetLastError());
    return BBC_OK;
}

// The original pair-side id of each tile item's anchor (items hold anchor ranks).
__global__ void k_item_anchors(const TileItem *__restrict__ items, int n, const int32_t *__restrict__ permS,
                               int32_t *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = permS[items[i].anchor];
}

bbc_status ensure_lists(bbc_graph *g, cudaStream_t st) {
    if (g->items_valid) return BBC_OK;
    const int sms = device_sm_count();
    Tuning T = resolve_tuning(nullptr, sms);
    T.split_wedges = auto_split(g->wedges, sms, T.blocks_per_sm);
    return build_work_lists(g, T, st);
}

}  // namespace
}  // namespace bbc

using namespace bbc;

extern "C" {

bbc_status bbc_cost_model_create(uint64_t seed, bbc_cost_model **out) {
    if (!out) {
        set_error("bbc_cost_model_create: NULL output");
        return BBC_E_INVALID_ARG;
    }
    *out = nullptr;
    try {
        BBC_TRY(check_device());
        bbc_cost_model *m = new bbc_cost_model();
        BBC_CUDA_TRY(cudaGetDevice(&m->device));
        std::vector<float> p(kParams, 0.f);
        uint64_t s = seed;
        auto uni = [&](float bound) {
            const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            return (float)((2.0 * u - 1.0) * bound);
        };
        // He-uniform weights, zero biases
        for (int i = 0; i < kH * kF; ++i) p[kOffW1 + i] = uni(std::sqrt(6.f / kF));
        for (int i = 0; i < kH * kH; ++i) p[kOffW2 + i] = uni(std::sqrt(6.f / kH));
        for (int i = 0; i < kH; ++i) p[kOffW3 + i] = uni(std::sqrt(6.f / kH));
        cudaError_t e = cudaMalloc(&m->params, kParams * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&m->grad, (kParams + 1) * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&m->m, kParams * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&m->v, kParams * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(m->params, p.data(), kParams * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(m->m, 0, kParams * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(m->v, 0, kParams * sizeof(float));
        if (e != cudaSuccess) {
            bbc_cost_model_free(m);
            return cuda_fail(e, "bbc_cost_model_create");
        }
        *out = m;
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_cost_model_create");
        return BBC_E_NO_MEMORY;
    }
}

void bbc_cost_model_free(bbc_cost_model *m) {
    if (!m) return;
    cudaFree(m->params);
    cudaFree(m->grad);
    cudaFree(m->m);
    cudaFree(m->v);
    delete m;
}

int32_t bbc_cost_model_num_params(void) { return kParams; }

bbc_status bbc_cost_model_get_params(const bbc_cost_model *m, float *host_out, int32_t capacity) {
    BBC_TRY(model_ready(m));
    if (!host_out || capacity < kParams) {
        set_error("bbc_cost_model_get_params: output smaller than the parameter count");
        return BBC_E_INVALID_ARG;
    }
    BBC_CUDA_TRY(cudaMemcpy(host_out, m->params, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    return BBC_OK;
}

bbc_status bbc_cost_model_set_params(bbc_cost_model *m, const float *host_in, int32_t n_params) {
    BBC_TRY(model_ready(m));
    if (!host_in || n_params != kParams) {
        set_error("bbc_cost_model_set_params: wrong parameter count");
        return BBC_E_INVALID_ARG;
    }
    BBC_CUDA_TRY(cudaMemcpy(m->params, host_in, kParams * sizeof(float), cudaMemcpyHostToDevice));
    BBC_CUDA_TRY(cudaMemset(m->m, 0, kParams * sizeof(float)));
    BBC_CUDA_TRY(cudaMemset(m->v, 0, kParams * sizeof(float)));
    m->step = 0;
    return BBC_OK;
}

bbc_status bbc_cost_model_loss_grad(bbc_cost_model *m, const float *X_dev, const float *t_dev, int32_t n,
                                    float *loss_host, float *grad_host, void *cuda_stream) {
    BBC_TRY(model_ready(m));
    if (n <= 0 || !X_dev || !t_dev || !loss_host) {
        set_error("bbc_cost_model_loss_grad: empty or NULL input");
        return BBC_E_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    BBC_CUDA_TRY(cudaMemsetAsync(m->grad, 0, (kParams + 1) * sizeof(float), st));
    note_launch();
    k_mlp_grad<<<grid_blocks(n), kWarpsPerBlock * 32, 0, st>>>(m->params, X_dev, t_dev, n, m->grad);
    BBC_CUDA_TRY(cudaGetLastError());
    std::vector<float> h(kParams + 1);
    BBC_CUDA_TRY(cudaMemcpyAsync(h.data(), m->grad, (kParams + 1) * sizeof(float), cudaMemcpyDeviceToHost, st));
    BBC_CUDA_TRY(cudaStreamSynchronize(st));
    *loss_host = h[kParams];
    if (grad_host) std::memcpy(grad_host, h.data(), kParams * sizeof(float));
    return BBC_OK;
}

bbc_status bbc_cost_model_fit(bbc_cost_model *m, const float *X_dev, const int64_t *cycles_dev, int32_t n,
                              int32_t steps, float lr, float *loss_host, void *cuda_stream) {
    BBC_TRY(model_ready(m));
    if (n <= 1 || !X_dev || !cycles_dev || steps < 0 || !(lr > 0.f)) {
        set_error("bbc_cost_model_fit: needs at least two samples, steps >= 0 and lr > 0");
        return BBC_E_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double *sums = nullptr;
    float *t = nullptr;
    BBC_TRY(dev_alloc_n(&sums, 2, st));
    bbc_status rc = dev_alloc_n(&t, (size_t)n, st);
    if (rc != BBC_OK) {
        dev_free(sums, st);
        return rc;
    }
    do {
        cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "bbc_cost_model_fit");
            break;
        }
        const auto cyc = reinterpret_cast<const long long *>(cycles_dev);
        note_launch();
        k_label_moments<<<std::min((n + 255) / 256, 1024), 256, 0, st>>>(cyc, n, sums);
        double hs[2] = {0, 0};
        e = cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "bbc_cost_model_fit");
            break;
        }
        const double mu = hs[0] / n, var = std::max(hs[1] / n - mu * mu, 1e-12);
        m->label_mu = (float)mu;
        m->label_sd = (float)std::sqrt(var);
        note_launch();
        k_labels<<<std::min((n + 255) / 256, 4096), 256, 0, st>>>(cyc, n, m->label_mu, m->label_sd, t);
        const float b1 = 0.9f, b2 = 0.999f;
        for (int s = 0; s < steps; ++s) {
            cudaMemsetAsync(m->grad, 0, (kParams + 1) * sizeof(float), st);
            note_launch();
            k_mlp_grad<<<grid_blocks(n), kWarpsPerBlock * 32, 0, st>>>(m->params, X_dev, t, n, m->grad);
            ++m->step;
            const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
            note_launch();
            k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(m->params, m->grad, m->m, m->v, kParams, lr, b1, b2,
                                                         1e-8f, c1, c2);
        }
        // the loss at the final parameters
        cudaMemsetAsync(m->grad, 0, (kParams + 1) * sizeof(float), st);
        note_launch();
        k_mlp_grad<<<grid_blocks(n), kWarpsPerBlock * 32, 0, st>>>(m->params, X_dev, t, n, m->grad);
        float lh = 0.f;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&lh, m->grad + kParams, sizeof lh, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "bbc_cost_model_fit");
            break;
        }
        if (loss_host) *loss_host = lh;
    } while (false);
    dev_free(t, st);
    dev_free(sums, st);
    return rc;
}

bbc_status bbc_cost_model_predict(const bbc_cost_model *m, const float *X_dev, int32_t n, float *y_dev,
                                  void *cuda_stream) {
    BBC_TRY(model_ready(m));
    if (n < 0 || (n > 0 && (!X_dev || !y_dev))) {
        set_error("bbc_cost_model_predict: NULL input or output");
        return BBC_E_INVALID_ARG;
    }
    if (n == 0) return BBC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    note_launch();
    k_mlp_predict<<<grid_blocks(n), kWarpsPerBlock * 32, 0, st>>>(m->params, X_dev, n, y_dev);
    BBC_CUDA_TRY(cudaGetLastError());
    return BBC_OK;
}

bbc_status bbc_item_features(bbc_graph *g, float *X_dev, int32_t capacity, int32_t *n_items, void *cuda_stream) {
    if (!g || !n_items || (capacity > 0 && !X_dev)) {
        set_error("bbc_item_features: NULL argument");
        return BBC_E_INVALID_ARG;
    }
    try {
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        BBC_TRY(ensure_lists(g, st));
        if (!X_dev && capacity == 0) {   // a query of the number of items
            *n_items = g->n_tile;
            return BBC_OK;
        }
        int n = 0;
        BBC_TRY(item_features(g, X_dev, capacity, &n, st));
        *n_items = n;
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_item_features");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_item_anchors(bbc_graph *g, int32_t *anchors_dev, int32_t capacity, int32_t *n_items,
                            void *cuda_stream) {
    if (!g || !n_items || (capacity > 0 && !anchors_dev)) {
        set_error("bbc_item_anchors: NULL argument");
        return BBC_E_INVALID_ARG;
    }
    try {
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        BBC_TRY(ensure_lists(g, st));
        *n_items = g->n_tile;
        if (g->n_tile > capacity) {
            set_error("bbc_item_anchors: capacity below the number of tile items");
            return BBC_E_INVALID_ARG;
        }
        if (g->n_tile == 0) return BBC_OK;
        note_launch();
        k_item_anchors<<<std::min((g->n_tile + 255) / 256, 4096), 256, 0, st>>>(g->tile_items, g->n_tile, g->permS,
                                                                              anchors_dev);
        BBC_CUDA_TRY(cudaGetLastError());
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_item_anchors");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_item_cycles(bbc_graph *g, int64_t *cycles_dev, int32_t capacity, int32_t *n_items,
                           void *cuda_stream) {
    if (!g || !n_items || (capacity > 0 && !cycles_dev)) {
        set_error("bbc_item_cycles: NULL argument");
        return BBC_E_INVALID_ARG;
    }
    try {
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        BBC_TRY(ensure_lists(g, st));
        *n_items = g->n_tile;
        if (g->n_tile > capacity) {
            set_error("bbc_item_cycles: capacity below the number of tile items");
            return BBC_E_INVALID_ARG;
        }
        BBC_CUDA_TRY(cudaMemsetAsync(g->totals, 0, 16, st));
        BBC_CUDA_TRY(cudaMemsetAsync(g->queue, 0, sizeof(QueueState), st));
        BBC_TRY(clear_centre_split(g, st));
        if (g->n_tile > 0) BBC_CUDA_TRY(cudaMemsetAsync(cycles_dev, 0, (size_t)g->n_tile * 8, st));
        DevGraph d = host_descriptor(g, false, true);
        BBC_CUDA_TRY(cudaMemcpyAsync(g->dgraph, &d, sizeof d, cudaMemcpyHostToDevice, st));
        CountLaunch L{};
        L.graphs = g->dgraph;
        L.tile_items = g->tile_items;
        L.n_tile_items = g->n_tile;
        L.queue = g->queue;
        L.tuning = g->items_tuning;
        L.prefetch = rows_exceed_l2(g);
        if (L.tuning.blocks_per_sm < 1) L.tuning.blocks_per_sm = 2;
        L.tuning.plain = 0;
        L.item_cycles = reinterpret_cast<long long *>(cycles_dev);
        BBC_TRY(launch_count(L, st));
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_item_cycles");
        return BBC_E_CUDA;
    }
}

bbc_status bbc_cost_model_order(const bbc_cost_model *m, bbc_graph *g, void *cuda_stream) {
    BBC_TRY(model_ready(m));
    if (!g) {
        set_error("bbc_cost_model_order: NULL graph");
        return BBC_E_INVALID_ARG;
    }
    try {
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        BBC_TRY(ensure_lists(g, st));
        const int n = g->n_tile;
        if (n <= 1) return BBC_OK;
        Buffers sc(st);
        float *X = nullptr, *y = nullptr;
        uint32_t *keys = nullptr, *idx = nullptr;
        TileItem *copy = nullptr;
        BBC_TRY(sc.get(&X, (size_t)n * kF));
        BBC_TRY(sc.get(&y, (size_t)n));
        BBC_TRY(sc.get(&keys, (size_t)n));
        BBC_TRY(sc.get(&idx, (size_t)n));
        BBC_TRY(sc.get(&copy, (size_t)n));
        int got = 0;
        BBC_TRY(item_features(g, X, n, &got, st));
        BBC_TRY(bbc_cost_model_predict(m, X, n, y, st));
        note_launch();
        k_order_keys<<<(n + 255) / 256, 256, 0, st>>>(y, n, keys, idx);
        BBC_TRY(radix_sort_pairs(keys, idx, n, 32, st));
        BBC_CUDA_TRY(cudaMemcpyAsync(copy, g->tile_items, (size_t)n * sizeof(TileItem), cudaMemcpyDeviceToDevice, st));
        note_launch();
        k_gather_tile_items<<<(n + 255) / 256, 256, 0, st>>>(copy, idx, n, g->tile_items);
        BBC_CUDA_TRY(cudaGetLastError());
        BBC_CUDA_TRY(cudaStreamSynchronize(st));
        g->layout_version++;   // captured batch plans hold copies of the old order
        return BBC_OK;
    } catch (...) {
        set_error("unexpected exception in bbc_cost_model_order");
        return BBC_E_CUDA;
    }
}

}  // extern "C"
