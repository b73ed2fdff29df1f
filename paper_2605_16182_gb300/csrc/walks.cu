// walks.cu -- causality-preserving temporal random walks (Tempest Sec. 2.1,
// 2.3, 2.4, 2.5).
//
// A hop at node v and time t reads v's group range [g0, g1) (two adjacent
// int32), binary-searches the group timestamps for the first group with
// ts > t (Gamma_t(v) = groups [c, g1)), draws the next edge with the walk's
// bias and reads one 16-byte entry.  Every draw comes from Philox keyed by
// (seed, walk, hop), so the result is independent of how walks are mapped to
// threads.
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
    double lam_hop, lam_start;
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

__global__ void __launch_bounds__(256) k_walks_full(const WalkView V, const WalkOut O)
{
    unsigned long long hops = 0, bytes = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < O.n_walks;
         w += (int64_t)gridDim.x * blockDim.x) {
        int32_t L = O.len_arr ? O.len_arr[w] : O.max_len;
        int bias = O.bias_arr ? (int)O.bias_arr[w] : O.bias;
        if (L < 2 || L > O.cap || bias < 0 || bias > 2) {
            // per-walk arrays that live on the device are checked here: the
            // walk is clamped into its row and the call reports EINVAL
            atomicOr(&O.cnt->status, 1ull);
            L = L < 2 ? 2 : (L > O.cap ? O.cap : L);
            bias = (bias < 0 || bias > 2) ? BIAS_UNIFORM : bias;
        }
        int32_t *nrow = O.node + w * (int64_t)O.cap;
        int64_t *trow = O.ts + w * (int64_t)O.cap;
        int32_t len = 0;
        if (V.m > 0) {
            // start edge (hop 0)
            Rand4 r = walk_rand(O.seed, (uint64_t)w, 0u);
            double u1 = u53(r.r0, r.r1);
            double u2 = u53(r.r2, r.r3);
            int64_t k;
            if (O.start_policy == TEMPEST_START_UNIFORM_EDGE) {
                k = uniform_index(u1, V.m);
            } else {
                const int64_t g = sampler_index(u1, V.G, bias, V.lam_start);
                const int64_t a = V.ts_goff[g];
                k = a + uniform_index(u2, (int64_t)V.ts_goff[g + 1] - a);
            }
            int32_t s = V.st_src[k], d = V.st_dst[k];
            const int64_t t0 = V.st_ts[k];
            if (!V.directed && (r.r3 & 1u)) {
                const int32_t x = s;
                s = d;
                d = x;
            }
            nrow[0] = s;
            nrow[1] = d;
            trow[0] = INT64_MIN;
            trow[1] = t0;
            len = 2;
            hops++;
            bytes += START_MODEL_BYTES;
            int32_t v = d;
            int64_t t = t0;
            for (uint32_t h = 1; len < L; h++) {
                const int32_t g0 = __ldg(V.gidx + v), g1 = __ldg(V.gidx + v + 1);
                const int32_t c = upper_bound_ts(V.ngts, g0, g1, t);
                if (c == g1) break;  // Gamma_t(v) is empty
                r = walk_rand(O.seed, (uint64_t)w, h);
                u1 = u53(r.r0, r.r1);
                int64_t idx;
                if (bias == BIAS_UNIFORM) {
                    const int32_t e0 = __ldg(V.ngo + c), e1 = __ldg(V.ngo + g1);
                    idx = e0 + uniform_index(u1, (int64_t)(e1 - e0));
                } else {
                    u2 = u53(r.r2, r.r3);
                    const int64_t j = sampler_index(u1, (int64_t)(g1 - c), bias, V.lam_hop);
                    const int32_t e0 = __ldg(V.ngo + c + j), e1 = __ldg(V.ngo + c + j + 1);
                    idx = e0 + uniform_index(u2, (int64_t)(e1 - e0));
                }
                const Entry e = V.ent[idx];
                nrow[len] = e.other;
                trow[len] = e.ts;
                hops++;
                bytes += hop_model_bytes((int64_t)(g1 - g0));
                v = e.other;
                t = e.ts;
                len++;
            }
        }
        for (int32_t i = len; i < O.cap; i++) {
            nrow[i] = -1;
            trow[i] = INT64_MIN;
        }
        O.len[w] = len;
    }
    hops = warp_sum(hops);
    bytes = warp_sum(bytes);
    if ((threadIdx.x & 31) == 0 && hops) {
        atomicAdd(&O.cnt->hops, hops);
        atomicAdd(&O.cnt->model_bytes, bytes);
    }
}

static WalkView make_view(tempest_t *h)
{
    WalkView V;
    V.st_src = h->st_src[h->cur].as<int32_t>();
    V.st_dst = h->st_dst[h->cur].as<int32_t>();
    V.st_ts = h->st_ts[h->cur].as<int64_t>();
    V.m = h->m;
    V.ts_goff = h->ts_goff.as<int32_t>();
    V.G = h->G;
    V.gidx = h->gidx.as<int32_t>();
    V.ngo = h->ngo.as<int32_t>();
    V.ngts = h->ngts.as<int64_t>();
    V.ent = h->ent.as<Entry>();
    V.directed = h->directed;
    V.lam_hop = h->lam_hop;
    V.lam_start = h->lam_start > 0.0 ? h->lam_start : (h->G > 0 ? 1.0 / (double)h->G : 1.0);
    return V;
}

int walks_run(tempest_t *h, const WalkRequest &rq)
{
    int rc;
    if ((rc = ensure(h, h->wcnt, sizeof(WalkCounters)))) return rc;
    cudaStream_t st = h->stream;
    cudaMemsetAsync(h->wcnt.p, 0, sizeof(WalkCounters), st);
    WalkView V = make_view(h);
    WalkOut O;
    O.n_walks = rq.n_walks;
    O.cap = rq.cap;
    O.max_len = rq.max_len;
    O.len_arr = rq.len_arr;
    O.bias = rq.bias;
    O.bias_arr = rq.bias_arr;
    O.start_policy = rq.start_policy;
    O.seed = rq.seed;
    O.node = rq.node;
    O.ts = rq.ts;
    O.len = rq.len;
    O.cnt = h->wcnt.as<WalkCounters>();
    int64_t launches = 0;
    if (rq.n_walks > 0) {
        int64_t grid = (rq.n_walks + 255) / 256;
        const int64_t cap = (int64_t)h->num_sms * 8;
        if (grid > cap) grid = cap;
        k_walks_full<<<(unsigned)grid, 256, 0, st>>>(V, O);
        launches++;
    }
    h->last_ws.n_walks = rq.n_walks;
    h->last_ws.launches = launches;
    return cuda_check(h, cudaGetLastError(), "walk launch");
}

}  // namespace tw
