// walkcore.cuh -- what every walk form shares: the device view of the index,
// the output description, the per-walk parameters, the start-edge draw, the
// hop draw and the per-hop traffic model (Tempest Sec. 2.1, 2.3, 2.5).
#pragma once

#include "engine.cuh"
#include "prims.cuh"

namespace tw {

// Slot of the Temporal Node2Vec pair table (csrc/pairs.cu): key = from << 32
// | to (undirected graphs: the smaller id first), cnt = live edges with that
// key; PAIR_EMPTY marks an unused slot.
struct alignas(16) PairSlot {
    unsigned long long key;
    int cnt;
    int pad;
};
constexpr unsigned long long PAIR_EMPTY = ~0ull;

__host__ __device__ __forceinline__ unsigned long long pair_key(int32_t a, int32_t b, int directed)
{
    if (!directed && b < a) {
        const int32_t x = a;
        a = b;
        b = x;
    }
    return (unsigned long long)(uint32_t)a << 32 | (uint32_t)b;
}

// Stafford's 64-bit finaliser ("Mix13"), the slot a key's probe starts at.
__host__ __device__ __forceinline__ uint64_t pair_hash(uint64_t k)
{
    k ^= k >> 30;
    k *= 0xbf58476d1ce4e5b9ull;
    k ^= k >> 27;
    k *= 0x94d049bb133111ebull;
    k ^= k >> 31;
    return k;
}

struct WalkView {
    // edge store, (ts, arrival) order: the live edges are [0, m) from these
    // pointers
    const int32_t *st_src;
    const int32_t *st_dst;
    const int64_t *st_ts;
    int64_t m;
    // timestamp-grouped view: group g starts at absolute store position tg[g]
    // (modulo 2^32) and ends where g + 1 starts; its live edges are store
    // offsets [max(tg[g] - s_lo, 0), tg[g + 1] - s_lo) with s_lo the absolute
    // position of the head (the head group may have lost a prefix)
    const int32_t *tg;
    uint32_t s_lo;
    int64_t G;
    // node view: record of node v (its groups, bucket base, first / last
    // group timestamps); group g's entries [ngo[g], ngo[g + 1]) in the pool
    const NodeRange *ngr;
    const int32_t *ngo;
    const int64_t *ngts;
    const Entry *ent;
    // time buckets of nodes with at least BKT_MIN_G groups (null: none)
    const int32_t *bkt;
    // active nodes in id order (PER_NODE starts; null when not built)
    const int32_t *pn_nodes;
    // per-node suffix sums of the group weights (weight-based bias; null when
    // not built)
    const double *gs;
    int bkt_log;
    int directed;
    // backward walks (the view is the in-view): searches run at t - 1 (the
    // last group earlier than t ends where the first group later than t - 1
    // begins), draws mirror the range, and back_swap walks a start edge from
    // its stored destination to its stored source
    int back, back_swap;
    ExpRate rate_hop, rate_start;
    // Temporal Node2Vec: live-pair table (null when not kept: q == 1) and the
    // factors 1/p, 1/q and beta_max = max(1/p, 1, 1/q)
    const PairSlot *pt;
    uint64_t pt_mask;
    double n2v_inv_p, n2v_inv_q, n2v_bmax;
};

// Store range [a, b) of timestamp group g (g < G).
__device__ __forceinline__ void ts_group_range(const WalkView &V, int64_t g, int64_t &a, int64_t &b)
{
    const int32_t x = (int32_t)((uint32_t)__ldg(V.tg + g) - V.s_lo);
    a = x > 0 ? x : 0;
    b = (int32_t)((uint32_t)__ldg(V.tg + g + 1) - V.s_lo);
}

struct WalkOut {
    int64_t n_walks;
    int32_t cap;
    int32_t max_len;
    const int32_t *len_arr;
    int bias;
    const uint8_t *bias_arr;
    int start_policy;
    int64_t pn_k;  // PER_NODE: walks per active node
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

// Time buckets of a node with G >= BKT_MIN_G groups [g0, g1) and first /
// last group timestamps tlo < thi (a node's groups have distinct
// timestamps).  A bucket is a run of 2^s time units aligned on absolute time
// (s chosen per node so that the node has about G >> log_b buckets): t lies
// in bucket (t >> s) - (tlo >> s) of the node, counted from the bucket of its
// first live group, a monotone map.  The node's table (at tb, K + 1 int32
// for its K buckets) holds for each bucket k the first group whose bucket is
// >= k, and g1 at k = K; entry 0 may name a group evicted since the table was
// built (the walker clamps it to g0).  Every group before table[k] is earlier
// than any t in bucket k and every group from table[k + 1] on is later, so
// for tlo <= t < thi the first group later than t lies in
// [max(table[k], g0), table[k + 1]], k = bucket(t).  Because buckets sit on
// absolute time, a table stays valid for the buckets a later state keeps, so
// each build copies those and fills only the buckets of new groups.
constexpr int32_t BKT_MIN_G = 32;
constexpr int32_t BKT_CHUNK = 1024;  // groups per table-fill task
constexpr int32_t BKT_HDR = 8;       // int32 header before a node's table (build bookkeeping)

// bucket of t relative to the node's first live group (tlo), width 2^s
__device__ __forceinline__ int32_t bkt_rel(int64_t t, int64_t tlo, int s) { return (int32_t)((t >> s) - (tlo >> s)); }

// The node record of v (two 16-byte loads of one sector).
__device__ __forceinline__ void load_range(const NodeRange *r, int32_t &g_lo, int32_t &g_hi, int32_t &tb,
                                           int64_t &t_first, int64_t &t_last, int32_t *bs = nullptr)
{
    const int4 a = __ldg(reinterpret_cast<const int4 *>(r));
    const longlong2 b = __ldg(reinterpret_cast<const longlong2 *>(r) + 1);
    g_lo = a.x;
    g_hi = a.y;
    tb = a.z;
    t_first = b.x;
    t_last = b.y;
    if (bs) *bs = a.w;
}

// Live groups [g0, g1) of v (the first 8 bytes of its record).
__device__ __forceinline__ void node_groups(const WalkView &V, int32_t v, int32_t &g0, int32_t &g1)
{
    const int2 a = __ldg(reinterpret_cast<const int2 *>(V.ngr + v));
    g0 = a.x;
    g1 = a.y;
}

// First group of v in [g0, g1) whose timestamp is > t (g1 when none):
// through the node's time buckets when it has them, else a plain bisection.
__device__ __forceinline__ int32_t first_later(const WalkView &V, int32_t v, int32_t g0, int32_t g1, int64_t t)
{
    if (V.bkt && g1 - g0 >= BKT_MIN_G) {
        int32_t a, b, tb, bs;
        int64_t tlo, thi;
        load_range(V.ngr + v, a, b, tb, tlo, thi, &bs);
        if (t < tlo) return g0;
        if (t >= thi) return g1;
        const int32_t k = bkt_rel(t, tlo, bs & 63);
        const int32_t lo = max(__ldg(V.bkt + tb + k), g0), hi = __ldg(V.bkt + tb + k + 1);
        return upper_bound_ts(V.ngts, lo, hi, t);
    }
    return upper_bound_ts(V.ngts, g0, g1, t);
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
    if (L < 2 || L > O.cap || bias < 0 || bias > 4) {
        atomicOr(&O.cnt->status, 1ull);
        L = L < 2 ? 2 : (L > O.cap ? O.cap : L);
        bias = (bias < 0 || bias > 4) ? BIAS_UNIFORM : bias;
    }
}

// Start draws and index-based hops treat the weight-based bias as the
// index-based exponential; a weight-based walk without weight sums (device
// bias arrays before the weights were enabled) reports EINVAL and walks as
// the index-based exponential.
constexpr int BIAS_EXP_WEIGHT = 3;
constexpr int BIAS_NODE2VEC = 4;
constexpr uint32_t N2V_MAX_TRIALS = 4096;
// The index sampler behind a bias: the weight-based and Node2Vec biases start
// (and Node2Vec proposes) like the index-based exponential.
__device__ __forceinline__ int start_bias(int bias) { return bias >= BIAS_EXP_WEIGHT ? BIAS_EXP : bias; }

__device__ __forceinline__ int hop_bias(const WalkView &V, int bias, WalkCounters *cnt)
{
    if (bias == BIAS_EXP_WEIGHT && !V.gs) {
        atomicOr(&cnt->status, 1ull);
        return BIAS_EXP;
    }
    return bias;
}

// Weight-based draw over the groups [c, g1) (Sec. 2.5): the smallest k with
// gs[k + 1] <= gs[c] (1 - u), i.e. the group whose running weight from c first
// reaches u gs[c] (k1: the 53-bit integer of u).
__device__ __forceinline__ int32_t weight_group(const WalkView &V, int32_t c, int32_t g1, uint64_t k1)
{
    const double R = __ldg(V.gs + c) * (1.0 - (double)k1 * 0x1.0p-53);
    int32_t lo = c, hi = g1 - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(V.gs + mid + 1) <= R) hi = mid;
        else lo = mid + 1;
    }
    return lo;
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
        if (V.back) k = V.m - 1 - k;
    } else {
        int64_t g = sampler_index_k(k1, V.G, start_bias(bias), V.rate_start);
        if (V.back) g = V.G - 1 - g;
        int64_t a, b;
        ts_group_range(V, g, a, b);
        k = V.back ? b - 1 - uniform_index_k(k2, b - a) : a + uniform_index_k(k2, b - a);
    }
    s = V.st_src[k];
    d = V.st_dst[k];
    t0 = V.st_ts[k];
    if (V.back_swap) {
        const int32_t x = s;
        s = d;
        d = x;
    }
    if (!V.directed && (r.r3 & 1u)) {
        const int32_t x = s;
        s = d;
        d = x;
    }
}

// Hop h >= 1 at a node whose groups are [c, g1) after the time filter: the
// drawn entry (uniform over the edges of Gamma_t(v), or a group by bias and
// then an edge inside it).
// (O: anything with the walk's seed and counters, .seed and .cnt.)
template <class OUT>
__device__ __forceinline__ Entry draw_entry(const WalkView &V, const OUT &O, int64_t w, uint32_t hop, int bias,
                                            int32_t c, int32_t g1)
{
    const Rand4 r = walk_rand(O.seed, (uint64_t)w, hop);
    const uint64_t h1 = u53_bits(r.r0, r.r1);
    int64_t idx;
    bias = hop_bias(V, bias, O.cnt);
    if (bias == BIAS_UNIFORM) {
        const int32_t e0 = __ldg(V.ngo + c), e1 = __ldg(V.ngo + g1);
        idx = e0 + uniform_index_k(h1, (int64_t)(e1 - e0));
    } else if (bias == BIAS_EXP_WEIGHT) {
        const uint64_t h2 = u53_bits(r.r2, r.r3);
        const int32_t k = weight_group(V, c, g1, h1);
        const int32_t e0 = __ldg(V.ngo + k), e1 = __ldg(V.ngo + k + 1);
        idx = e0 + uniform_index_k(h2, (int64_t)(e1 - e0));
    } else {
        const uint64_t h2 = u53_bits(r.r2, r.r3);
        const int64_t j = sampler_index_k(h1, (int64_t)(g1 - c), start_bias(bias), V.rate_hop);
        const int32_t e0 = __ldg(V.ngo + c + j), e1 = __ldg(V.ngo + c + j + 1);
        idx = e0 + uniform_index_k(h2, (int64_t)(e1 - e0));
    }
    return V.ent[idx];
}

// Backward hop at a node whose groups earlier than t are [g0, c), in the
// mirrored order: uniform over the edges (position last - q), or group
// c - 1 - j by the bias, then an edge of it (position last - q).
template <class OUT>
__device__ __forceinline__ Entry draw_entry_back(const WalkView &V, const OUT &O, int64_t w, uint32_t hop,
                                                 int bias, int32_t g0, int32_t c)
{
    const Rand4 r = walk_rand(O.seed, (uint64_t)w, hop);
    const uint64_t h1 = u53_bits(r.r0, r.r1);
    int64_t idx;
    bias = hop_bias(V, bias, O.cnt);  // no weight sums backward: flagged
    if (bias == BIAS_UNIFORM) {
        const int32_t e0 = __ldg(V.ngo + g0), e1 = __ldg(V.ngo + c);
        idx = e1 - 1 - uniform_index_k(h1, (int64_t)(e1 - e0));
    } else {
        const uint64_t h2 = u53_bits(r.r2, r.r3);
        const int64_t j = sampler_index_k(h1, (int64_t)(c - g0), start_bias(bias), V.rate_hop);
        const int32_t gg = c - 1 - (int32_t)j;
        const int32_t e0 = __ldg(V.ngo + gg), e1 = __ldg(V.ngo + gg + 1);
        idx = e1 - 1 - uniform_index_k(h2, (int64_t)(e1 - e0));
    }
    return V.ent[idx];
}

// Temporal Node2Vec factor beta(u, w) of candidate w from a node whose
// predecessor on the walk is u >= 0 (Sec. 2.5): 1/p when w is u, 1 when w is
// a neighbour of u (a live edge u -> w; w -> u for backward walks, which walk
// the time-reversed graph; either orientation undirected), 1/q otherwise.
// `lookups` counts pair-table tests; a missing table (device per-walk biases
// before tempest_set_node2vec kept one) is flagged and reads as no neighbour.
__device__ __forceinline__ double n2v_beta(const WalkView &V, WalkCounters *cnt, int32_t u, int32_t w,
                                           int &lookups)
{
    if (w == u) return V.n2v_inv_p;
    if (V.n2v_inv_q == 1.0) return 1.0;  // neighbour or not, the factor is 1
    lookups++;
    if (!V.pt) {
        atomicOr(&cnt->status, 1ull);
        return V.n2v_inv_q;
    }
    const unsigned long long key = V.back ? pair_key(w, u, V.directed) : pair_key(u, w, V.directed);
    uint64_t s = pair_hash(key) & V.pt_mask;
    for (uint64_t i = 0; i <= V.pt_mask; i++, s = (s + 1) & V.pt_mask) {
        const PairSlot e = V.pt[s];
        if (e.key == key) return e.cnt > 0 ? 1.0 : V.n2v_inv_q;
        if (e.key == PAIR_EMPTY) break;
    }
    return V.n2v_inv_q;
}

// Whether proposal k of a Node2Vec hop with factor beta is accepted: always
// when beta is beta_max, else when u * beta_max < beta for the uniform u of
// Philox word 1 = 2^31 + k (the comparison is exact in double, as in the
// oracle).
__device__ __forceinline__ bool n2v_accept(const WalkView &V, uint64_t seed, uint64_t w, uint32_t hop, uint32_t k,
                                           double beta)
{
    if (beta >= V.n2v_bmax) return true;
    const Rand4 a = walk_rand2(seed, w, hop, 0x80000000u | k);
    return (double)u53_bits(a.r0, a.r1) * 0x1.0p-53 * V.n2v_bmax < beta;
}

// Proposal k of a Node2Vec hop over the candidate groups (forward [c, g1),
// backward [g0, c) mirrored): the exponential sampler's group, then an edge
// uniformly inside it, from Philox word 1 = k.
__device__ __forceinline__ Entry n2v_propose(const WalkView &V, uint64_t seed, uint64_t w, uint32_t hop, uint32_t k,
                                             int32_t g0, int32_t c, int32_t g1)
{
    const Rand4 r = walk_rand2(seed, w, hop, k);
    const uint64_t h1 = u53_bits(r.r0, r.r1), h2 = u53_bits(r.r2, r.r3);
    const int32_t lo = V.back ? g0 : c, hi = V.back ? c : g1;
    const int32_t j = (int32_t)sampler_index_k(h1, (int64_t)(hi - lo), BIAS_EXP, V.rate_hop);
    const int32_t gg = V.back ? hi - 1 - j : lo + j;
    const int32_t e0 = __ldg(V.ngo + gg), e1 = __ldg(V.ngo + gg + 1);
    const int64_t q = uniform_index_k(h2, (int64_t)(e1 - e0));
    return V.ent[V.back ? (int64_t)e1 - 1 - q : (int64_t)e0 + q];
}

// One Node2Vec hop by rejection (Sec. 2.5); u < 0 (a PER_NODE start, no
// predecessor) takes the first proposal.  False when N2V_MAX_TRIALS
// proposals were all rejected (the walk ends).  bytes adds the sector model
// of the extra reads: 12 + 16 per proposal after the first, 32 per lookup.
template <class OUT>
__device__ __forceinline__ bool draw_n2v(const WalkView &V, const OUT &O, int64_t w, uint32_t hop, int32_t g0,
                                         int32_t c, int32_t g1, int32_t u, Entry &out, unsigned long long &bytes)
{
    for (uint32_t k = 0; k < N2V_MAX_TRIALS; k++) {
        const Entry e = n2v_propose(V, O.seed, (uint64_t)w, hop, k, g0, c, g1);
        if (k > 0) bytes += 12 + 16;
        if (u < 0) {
            out = e;
            return true;
        }
        int lk = 0;
        const double beta = n2v_beta(V, O.cnt, u, e.other, lk);
        bytes += 32ull * (unsigned)lk;
        if (n2v_accept(V, O.seed, (uint64_t)w, hop, k, beta)) {
            out = e;
            return true;
        }
    }
    return false;
}

// Padding of one walk output row (node -1, ts INT64_MIN) from cell l to the
// row end, by the whole warp on consecutive cells, with 16-byte stores where
// the row layout allows (vec); streaming stores, as nothing reads padding back
// during a walk call.
__device__ __forceinline__ void warp_pad_row(int32_t *nr, int64_t *tr, int32_t l, int32_t cap, int lane, bool vec)
{
    l = l < 0 ? 0 : l;
    if (vec) {
        const int4 n4 = make_int4(-1, -1, -1, -1);
        const longlong2 t2 = make_longlong2(INT64_MIN, INT64_MIN);
        for (int32_t q = (l >> 2) + lane; q < (cap >> 2); q += 32) {
            if (4 * q >= l) {
                __stcs(reinterpret_cast<int4 *>(nr) + q, n4);
            } else {
                for (int32_t i = l; i < 4 * q + 4; i++) nr[i] = -1;
            }
        }
        for (int32_t q = (l >> 1) + lane; q < (cap >> 1); q += 32) {
            if (2 * q >= l) __stcs(reinterpret_cast<longlong2 *>(tr) + q, t2);
            else tr[l] = INT64_MIN;  // l odd: the second half of the pair
        }
    } else {
        for (int32_t i = l + lane; i < cap; i += 32) {
            nr[i] = -1;
            tr[i] = INT64_MIN;
        }
    }
}

__device__ __forceinline__ bool pad_vec_ok(const int32_t *node, const int64_t *ts, int32_t cap)
{
    return (cap & 3) == 0 && ((uintptr_t)node & 15) == 0 && ((uintptr_t)ts & 15) == 0;
}

// Padding of the rows of the warp's lanes: lane i names walk w (< 0: none)
// and the cell its padding starts at (from >= cap: none); rows are written
// one at a time by the whole warp.  Every lane of the warp must call it.
__device__ __forceinline__ void warp_pad_walk_rows(int32_t *node, int64_t *ts, int32_t cap, int64_t w, int32_t from,
                                                   int lane)
{
    const bool vec = pad_vec_ok(node, ts, cap);
    unsigned todo = __ballot_sync(0xffffffffu, w >= 0 && from < cap);
    while (todo) {
        const int r = __ffs(todo) - 1;
        todo &= todo - 1;
        const int64_t wr = __shfl_sync(0xffffffffu, w, r);
        const int32_t l = __shfl_sync(0xffffffffu, from, r);
        warp_pad_row(node + wr * (int64_t)cap, ts + wr * (int64_t)cap, l, cap, lane, vec);
    }
}

// The time a walk searches at after reaching a node at time t (forward: t;
// backward: t - 1), and before its first hop under PER_NODE.
__device__ __forceinline__ int64_t search_time(const WalkView &V, int64_t t) { return V.back ? t - 1 : t; }
__device__ __forceinline__ int64_t pernode_time(const WalkView &V) { return V.back ? INT64_MAX - 1 : INT64_MIN; }

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
    int64_t pn_k;  // PER_NODE: walks per active node
};

WalkView make_view(tempest_t *h, int back = 0);
// Node2Vec fields of a view from the handle that keeps the pair table
void view_n2v(WalkView &V, const tempest_t *h);
// One persistent streaming launch over n_req requests of one direction whose
// descriptors are in device memory; counters in cnt (zeroed here unless
// clear is false, when the launch adds to them).
// may_n2v: a request may take the Node2Vec bias (a per-walk bias array, or
// that scalar bias).
int walks_multi_launch(tempest_t *h, int direction, const ReqDesc *dev_reqs, int n_req, int64_t total,
                       WalkCounters *cnt, cudaStream_t st, bool clear = true, bool may_n2v = true);
int coop_run(tempest_t *h, const WalkView &V, const WalkOut &O, int64_t &launches);
int graph_run(tempest_t *h, const WalkView &V, const WalkOut &O, int64_t &launches);

}  // namespace tw
