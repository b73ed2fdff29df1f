// walkcore.cuh -- what every walk form shares: the device view of the index,
// the output description, the per-walk parameters, the start-edge draw, the
// hop draw and the per-hop traffic model (Tempest Sec. 2.1, 2.3, 2.5).
#pragma once

#include "engine.cuh"
#include "prims.cuh"

namespace tw {

struct WalkView {
    // edge store, (ts, arrival) order
    const int32_t *st_src;
    const int32_t *st_dst;
    const int64_t *st_ts;
    int64_t m;
    // timestamp-grouped view
    const int32_t *ts_goff;
    int64_t G;
    // node view
    const int32_t *gidx;   // [N+1]
    const int32_t *ngo;    // [Gn+1]
    const int64_t *ngts;   // [Gn]
    const Entry *ent;      // [M]
    int directed;
    ExpRate rate_hop, rate_start;
};

struct WalkOut {
    int64_t n_walks;
    int32_t cap;
    int32_t max_len;
    const int32_t *len_arr;
    int bias;
    const uint8_t *bias_arr;
    int start_policy;
    uint64_t seed;
    int32_t *node;
    int64_t *ts;
    int32_t *len;
    WalkCounters *cnt;
};

// first index in [lo, hi) whose group timestamp is > t
__device__ __forceinline__ int32_t upper_bound_ts(const int64_t *__restrict__ gts, int32_t lo, int32_t hi,
                                                  int64_t t)
{
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(gts + mid) > t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int ceil_log2_plus1(int64_t G)
{
    // ceil(log2(G + 1)) for G >= 0
    return 64 - __clzll((unsigned long long)G);
}

// Sector model of one hop's traffic at a node with G groups: range read,
// binary search (last two levels share a sector), chosen entry, output write
// (node + ts) and walk state read + write.
__device__ __forceinline__ unsigned long long hop_model_bytes(int64_t G)
{
    int s = ceil_log2_plus1(G) - 2;
    if (s < 1) s = 1;
    return 32ull * (unsigned long long)(1 + s + 1) + 12ull + 16ull;
}
constexpr unsigned long long START_MODEL_BYTES = 3 * 32 + 4 + 4 + 8 + 8 + 4;


// Per-walk length cap and bias.  Arrays that live on the device are checked
// here: an out-of-range value is clamped into the walk's row and the call
// reports EINVAL through the status word.
__device__ __forceinline__ void walk_params(const WalkOut &O, int64_t w, int32_t &L, int &bias)
{
    L = O.len_arr ? O.len_arr[w] : O.max_len;
    bias = O.bias_arr ? (int)O.bias_arr[w] : O.bias;
    if (L < 2 || L > O.cap || bias < 0 || bias > 2) {
        atomicOr(&O.cnt->status, 1ull);
        L = L < 2 ? 2 : (L > O.cap ? O.cap : L);
        bias = (bias < 0 || bias > 2) ? BIAS_UNIFORM : bias;
    }
}

// Hop 0: the start edge (s -> d at t0), oriented for undirected graphs.
__device__ __forceinline__ void start_edge(const WalkView &V, const WalkOut &O, int64_t w, int bias, int32_t &s,
                                           int32_t &d, int64_t &t0)
{
    const Rand4 r = walk_rand(O.seed, (uint64_t)w, 0u);
    const uint64_t k1 = u53_bits(r.r0, r.r1);
    const uint64_t k2 = u53_bits(r.r2, r.r3);
    int64_t k;
    if (O.start_policy == TEMPEST_START_UNIFORM_EDGE) {
        k = uniform_index_k(k1, V.m);
    } else {
        const int64_t g = sampler_index_k(k1, V.G, bias, V.rate_start);
        const int64_t a = V.ts_goff[g];
        k = a + uniform_index_k(k2, (int64_t)V.ts_goff[g + 1] - a);
    }
    s = V.st_src[k];
    d = V.st_dst[k];
    t0 = V.st_ts[k];
    if (!V.directed && (r.r3 & 1u)) {
        const int32_t x = s;
        s = d;
        d = x;
    }
}

// Hop h >= 1 at a node whose groups are [c, g1) after the time filter: the
// drawn entry (uniform over the edges of Gamma_t(v), or a group by bias and
// then an edge inside it).
__device__ __forceinline__ Entry draw_entry(const WalkView &V, const WalkOut &O, int64_t w, uint32_t hop, int bias,
                                            int32_t c, int32_t g1)
{
    const Rand4 r = walk_rand(O.seed, (uint64_t)w, hop);
    const uint64_t h1 = u53_bits(r.r0, r.r1);
    int64_t idx;
    if (bias == BIAS_UNIFORM) {
        const int32_t e0 = __ldg(V.ngo + c), e1 = __ldg(V.ngo + g1);
        idx = e0 + uniform_index_k(h1, (int64_t)(e1 - e0));
    } else {
        const uint64_t h2 = u53_bits(r.r2, r.r3);
        const int64_t j = sampler_index_k(h1, (int64_t)(g1 - c), bias, V.rate_hop);
        const int32_t e0 = __ldg(V.ngo + c + j), e1 = __ldg(V.ngo + c + j + 1);
        idx = e0 + uniform_index_k(h2, (int64_t)(e1 - e0));
    }
    return V.ent[idx];
}

// One walk request of a multi-request launch (device copy).  offset is the
// first global walk id of the request inside the launch.
struct ReqDesc {
    int64_t n_walks;
    int64_t offset;
    const int32_t *len_arr;
    const uint8_t *bias_arr;
    int32_t *node;
    int64_t *ts;
    int32_t *len;
    uint64_t seed;
    int32_t cap;
    int32_t max_len;
    int32_t bias;
    int32_t start_policy;
};

WalkView make_view(tempest_t *h);
// One persistent streaming launch (plus row padding) over n_req requests
// whose descriptors are in device memory; counters in cnt (zeroed here).
int walks_multi_launch(tempest_t *h, const ReqDesc *dev_reqs, int n_req, int64_t total, WalkCounters *cnt,
                       cudaStream_t st);
int coop_run(tempest_t *h, const WalkView &V, const WalkOut &O, int64_t &launches);
int graph_run(tempest_t *h, const WalkView &V, const WalkOut &O, int64_t &launches);

}  // namespace tw
