// walks.cu -- causality-preserving temporal random walks (Tempest Sec. 2.1,
// 2.3, 2.4, 2.5).
//
// A hop at node v and time t reads v's group range [g0, g1) (two adjacent
// int32), binary-searches the group timestamps for the first group with
// ts > t (Gamma_t(v) = groups [c, g1)), draws the next edge with the walk's
// bias and reads one 16-byte entry.  Every draw comes from Philox keyed by
// (seed, walk, hop), so the result is independent of how walks are mapped to
// threads.
#include <algorithm>
#include <type_traits>

#include "engine.cuh"
#include "prims.cuh"
#include "walkcore.cuh"

namespace tw {

__global__ void __launch_bounds__(256) k_walks_full(const WalkView V, const WalkOut O)
{
    unsigned long long hops = 0, bytes = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < O.n_walks;
         w += (int64_t)gridDim.x * blockDim.x) {
        int32_t L = O.len_arr ? O.len_arr[w] : O.max_len;
        int bias = O.bias_arr ? (int)O.bias_arr[w] : O.bias;
        if (L < 2 || L > O.cap || bias < 0 || bias > 4) {
            // per-walk arrays that live on the device are checked here: the
            // walk is clamped into its row and the call reports EINVAL
            atomicOr(&O.cnt->status, 1ull);
            L = L < 2 ? 2 : (L > O.cap ? O.cap : L);
            bias = (bias < 0 || bias > 4) ? BIAS_UNIFORM : bias;
        }
        int32_t *nrow = O.node + w * (int64_t)O.cap;
        int64_t *trow = O.ts + w * (int64_t)O.cap;
        int32_t len = 0;
        if (V.m > 0) {
            int32_t v;
            int32_t u = -1;  // the node before v (Node2Vec); none at a PER_NODE start
            int64_t t;
            Rand4 r;
            if (O.start_policy == TEMPEST_START_PER_NODE) {
                // the walk starts at an active node before every live edge
                v = __ldg(V.pn_nodes + w / O.pn_k);
                t = pernode_time(V);
                nrow[0] = v;
                trow[0] = INT64_MIN;
                len = 1;
            } else {
                // start edge (hop 0)
                r = walk_rand(O.seed, (uint64_t)w, 0u);
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
                int32_t s = V.st_src[k], d = V.st_dst[k];
                const int64_t t0 = V.st_ts[k];
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
                nrow[0] = s;
                nrow[1] = d;
                trow[0] = INT64_MIN;
                trow[1] = t0;
                len = 2;
                hops++;
                bytes += START_MODEL_BYTES;
                u = s;
                v = d;
                t = search_time(V, t0);
            }
            while (len < L) {
                const uint32_t h = (uint32_t)(len - 1);  // counter of the draw for position len
                int32_t g0, g1;
                node_groups(V, v, g0, g1);
                const int32_t c = first_later(V, v, g0, g1, t);
                if (V.back ? c == g0 : c == g1) break;  // Gamma_t(v) is empty
                if (V.back || bias == BIAS_NODE2VEC) {
                    Entry e;
                    if (bias == BIAS_NODE2VEC) {
                        if (!draw_n2v(V, O, w, h, g0, c, g1, u, e, bytes)) break;  // all proposals rejected
                    } else {
                        e = draw_entry_back(V, O, w, h, bias, g0, c);
                    }
                    nrow[len] = e.other;
                    trow[len] = e.ts;
                    hops++;
                    bytes += hop_model_bytes((int64_t)(g1 - g0));
                    u = v;
                    v = e.other;
                    t = search_time(V, e.ts);
                    len++;
                    continue;
                }
                r = walk_rand(O.seed, (uint64_t)w, h);
                const uint64_t h1 = u53_bits(r.r0, r.r1);
                int64_t idx;
                const int hb = hop_bias(V, bias, O.cnt);
                if (hb == BIAS_UNIFORM) {
                    const int32_t e0 = __ldg(V.ngo + c), e1 = __ldg(V.ngo + g1);
                    idx = e0 + uniform_index_k(h1, (int64_t)(e1 - e0));
                } else if (hb == BIAS_EXP_WEIGHT) {
                    const uint64_t h2 = u53_bits(r.r2, r.r3);
                    const int32_t kg = weight_group(V, c, g1, h1);
                    const int32_t e0 = __ldg(V.ngo + kg), e1 = __ldg(V.ngo + kg + 1);
                    idx = e0 + uniform_index_k(h2, (int64_t)(e1 - e0));
                } else {
                    const uint64_t h2 = u53_bits(r.r2, r.r3);
                    const int64_t j = sampler_index_k(h1, (int64_t)(g1 - c), start_bias(hb), V.rate_hop);
                    const int32_t e0 = __ldg(V.ngo + c + j), e1 = __ldg(V.ngo + c + j + 1);
                    idx = e0 + uniform_index_k(h2, (int64_t)(e1 - e0));
                }
                const Entry e = V.ent[idx];
                nrow[len] = e.other;
                trow[len] = e.ts;
                hops++;
                bytes += hop_model_bytes((int64_t)(g1 - g0));
                u = v;
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

// ---------------------------------------------------------------------------
// Streaming walker.
//
// Each lane runs a small state machine and carries one walk at a time; every
// loop iteration consumes the values loaded in the previous iteration,
// computes, and issues the next (at most three independent) loads.  A lane
// whose walk ends takes the next walk id from a warp-aggregated atomic
// counter at once, so lanes never wait for the longest walk of their warp
// and every iteration keeps one memory round trip in flight per lane.
//
// The search for c = the first group of v with ts > t uses interpolation on
// the group timestamps (arrival times are close to uniform inside a node's
// range, so O(log log G) probes), falling back to a bisection probe whenever
// a probe did not halve the bracket (at most ~2 log2 G probes).  Any exact
// search returns the same c as the plain binary search.
// ---------------------------------------------------------------------------
enum : int {
    S_FETCH = 0,   // needs a walk
    S_NEW,         // walk assigned: draw the start
    S_PNODE,       // PER_NODE: start node loaded
    S_SGROUP,      // start timestamp group offsets loaded
    S_EDGE,        // start edge loaded
    S_RANGE,       // node record loaded (groups, bucket base, first / last ts)
    S_BKT,         // time-bucket table pair loaded (high-degree node)
    S_SEARCH,      // one probe loaded
    S_WTOT,        // weight of Gamma loaded (weight-based bias)
    S_WSEARCH,     // one suffix sum loaded (weight-based bias)
    S_PICK2,       // chosen group's entry range loaded
    S_HOP,         // chosen entry loaded
    S_N2V,         // Node2Vec: one pair-table slot loaded
    S_EXIT
};

struct SmLane {
    int64_t w;
    int64_t t;       // current time
    int64_t vL, vR;  // bracket values: a[L] <= t < a[R]
    uint64_t ud;     // saved 53-bit uniform for the draw inside a range
    int32_t L, R;    // bracket
    int32_t g0, g1;  // group range of the current node
    int32_t v;       // current node
    int32_t len, cap_len;
    int32_t state;
    int32_t bias;
    int32_t prev_w;  // bracket width before the last probe (Node2Vec: probes of the pair table)
    uint32_t hop;
    uint32_t orient;  // start: orientation bit; Node2Vec: proposal number of the hop
    int32_t u;        // the node before v (Node2Vec); -1 at a PER_NODE start
};

__device__ __forceinline__ int32_t interp_probe(int32_t L, int32_t R, int64_t vL, int64_t vR, int64_t t,
                                                bool bisect)
{
    // L < R - 1, vL <= t < vR.  The guess only steers the search (the
    // comparison against t is exact), so single precision is enough.
    if (bisect) return L + ((R - L) >> 1);
    // scale both differences into 31 bits so that only 32-bit integer to
    // float conversions are needed (64-bit ones issue on the FP64 pipe)
    const uint64_t d = (uint64_t)vR - (uint64_t)vL;
    const uint64_t a = (uint64_t)t - (uint64_t)vL;
    const int sh = max(0, 33 - __clzll((long long)d));
    const float f = __fdividef((float)(uint32_t)(a >> sh), (float)(uint32_t)(d >> sh));
    int32_t p = L + 1 + (int32_t)(f * (float)(R - L - 1));
    if (p <= L) p = L + 1;
    if (p >= R) p = R - 1;
    return p;
}

// A provider maps a global walk id g in [0, total()) to a walk of some
// request: its own walk number (which keys its Philox stream), its seed,
// start policy, output row and length slot.
struct OneReq {
    WalkOut O;
    struct Ctx {
        int64_t w;
    };
    __device__ __forceinline__ int64_t total() const { return O.n_walks; }
    __device__ __forceinline__ void open(int64_t g, Ctx &c, int32_t &L, int &bias) const
    {
        c.w = g;
        walk_params(O, g, L, bias);
    }
    __device__ __forceinline__ uint64_t seed(const Ctx &) const { return O.seed; }
    __device__ __forceinline__ uint64_t wid(const Ctx &c) const { return (uint64_t)c.w; }
    __device__ __forceinline__ int policy(const Ctx &) const { return O.start_policy; }
    __device__ __forceinline__ int32_t *nrow(const Ctx &c) const { return O.node + c.w * (int64_t)O.cap; }
    __device__ __forceinline__ int64_t *trow(const Ctx &c) const { return O.ts + c.w * (int64_t)O.cap; }
    __device__ __forceinline__ void finish(const Ctx &c, int32_t len) const { O.len[c.w] = len; }
    __device__ __forceinline__ int32_t cap(const Ctx &) const { return O.cap; }
    __device__ __forceinline__ int64_t pn_k(const Ctx &) const { return O.pn_k; }
    __device__ __forceinline__ WalkCounters *cnt() const { return O.cnt; }
};

struct ManyReq {
    const ReqDesc *reqs;  // sorted by offset, reqs[0].offset == 0
    int n_req;
    int64_t total_;
    WalkCounters *counters;
    struct Ctx {
        int64_t w;
        int32_t r;
    };
    __device__ __forceinline__ int64_t total() const { return total_; }
    __device__ __forceinline__ void open(int64_t g, Ctx &c, int32_t &L, int &bias) const
    {
        int lo = 0, hi = n_req - 1;  // last request whose offset <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (reqs[mid].offset <= g) lo = mid;
            else hi = mid - 1;
        }
        const ReqDesc &q = reqs[lo];
        c.r = lo;
        c.w = g - q.offset;
        if (c.w < 0 || c.w >= q.n_walks) {  // corrupt request table
            atomicOr(&counters->status, 1ull << 8);
            c.w = 0;
        }
        L = q.len_arr ? q.len_arr[c.w] : q.max_len;
        bias = q.bias_arr ? (int)q.bias_arr[c.w] : q.bias;
        if (L < 2 || L > q.cap || bias < 0 || bias > 4) {
            atomicOr(&counters->status, 1ull);
            L = L < 2 ? 2 : (L > q.cap ? q.cap : L);
            bias = (bias < 0 || bias > 4) ? BIAS_UNIFORM : bias;
        }
    }
    __device__ __forceinline__ uint64_t seed(const Ctx &c) const { return reqs[c.r].seed; }
    __device__ __forceinline__ uint64_t wid(const Ctx &c) const { return (uint64_t)c.w; }
    __device__ __forceinline__ int policy(const Ctx &c) const { return reqs[c.r].start_policy; }
    __device__ __forceinline__ int32_t *nrow(const Ctx &c) const
    {
        return reqs[c.r].node + c.w * (int64_t)reqs[c.r].cap;
    }
    __device__ __forceinline__ int64_t *trow(const Ctx &c) const
    {
        return reqs[c.r].ts + c.w * (int64_t)reqs[c.r].cap;
    }
    __device__ __forceinline__ void finish(const Ctx &c, int32_t len) const { reqs[c.r].len[c.w] = len; }
    __device__ __forceinline__ int32_t cap(const Ctx &c) const { return reqs[c.r].cap; }
    __device__ __forceinline__ int64_t pn_k(const Ctx &c) const { return reqs[c.r].pn_k; }
    __device__ __forceinline__ WalkCounters *cnt() const { return counters; }
};

// MINB: resident CTAs per SM the register budget is cut for (4: 64
// registers; 5: 48 registers with a few spills, for more warps in flight).
// BACK: backward walks (the view is the in-view; a compile-time copy of
// V.back, so forward walks carry no direction tests).
// N2V: whether the Temporal Node2Vec rejection states are compiled in (they
// cost registers); without them a Node2Vec walk takes its first proposal,
// which is exactly the walk when p = q = 1 (every beta is beta_max) and is
// flagged otherwise.
template <class P, int MINB, bool N2V, bool BACK>
__global__ void __launch_bounds__(256, MINB) k_walks_stream(const WalkView V, const P Pv,
                                                             unsigned long long *next_walk)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    SmLane s;
    typename P::Ctx cx;
    s.state = S_FETCH;
    s.w = 0;
    int64_t y0 = 0;           // loaded 64-bit value
    int32_t z0 = 0, z1 = 0;   // loaded 32-bit values
    int32_t z2 = 0, z3 = 0;  // z3: the node record's bucket width word
    int64_t y1 = 0;
    unsigned long long hops = 0, bytes = 0;
    const int64_t N = Pv.total();

    // warp-local queue of walk ids [q_next, q_end), refilled WALK_CHUNK at a
    // time from the global counter (warp-uniform values)
    constexpr int64_t WALK_CHUNK = 256;
    int64_t q_next = 0, q_end = 0;
    while (true) {
        // lanes without a walk take the next ids from the warp's queue
        unsigned need = __ballot_sync(0xffffffffu, s.state == S_FETCH);
        while (need) {
            if (q_next >= q_end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(next_walk, (unsigned long long)WALK_CHUNK);
                base = __shfl_sync(0xffffffffu, base, 0);
                if ((int64_t)base >= N) {
                    if (s.state == S_FETCH) s.state = S_EXIT;
                    break;
                }
                q_next = (int64_t)base;
                q_end = min(N, q_next + WALK_CHUNK);
            }
            const int64_t avail = q_end - q_next;
            const int rank = __popc(need & lt);
            const int take = (int)min((int64_t)__popc(need), avail);
            if (s.state == S_FETCH && rank < take) {
                s.w = q_next + rank;
                s.state = S_NEW;
            }
            q_next += take;
            need = __ballot_sync(0xffffffffu, s.state == S_FETCH);
        }
        if (__all_sync(0xffffffffu, s.state == S_EXIT)) break;

        bool pick = false;   // the bracket closed this iteration: draw now
        bool finish = false; // the walk ended this iteration

        // the chosen entry (z0 other, y0 ts) becomes position len
        auto commit_hop = [&]() {
            Pv.nrow(cx)[s.len] = z0;
            Pv.trow(cx)[s.len] = y0;
            hops++;
            bytes += hop_model_bytes((int64_t)(s.g1 - s.g0));
            s.len++;
            s.hop++;
            if (N2V) s.u = s.v;
            s.v = z0;
            s.t = (BACK ? y0 - 1 : y0);
            if (s.len >= s.cap_len) {
                finish = true;
            } else {
                load_range(V.ngr + z0, z0, z1, z2, y0, y1, &z3);
                s.state = S_RANGE;
            }
        };
        // Node2Vec proposal s.orient of this hop (candidate groups from c =
        // s.R): loads the chosen group's entry range
        auto n2v_issue = [&]() {
            const Rand4 r = walk_rand2(Pv.seed(cx), Pv.wid(cx), s.hop, s.orient);
            s.ud = u53_bits(r.r2, r.r3);
            const int32_t lo = BACK ? s.g0 : s.R, hi = BACK ? s.R : s.g1;
            const int32_t j = (int32_t)sampler_index_k(u53_bits(r.r0, r.r1), (int64_t)(hi - lo), BIAS_EXP, V.rate_hop);
            const int32_t gg = BACK ? hi - 1 - j : lo + j;
            z0 = __ldg(V.ngo + gg);
            z1 = __ldg(V.ngo + gg + 1);
            s.state = S_PICK2;
        };
        // accept the loaded proposal with factor beta, or draw the next one
        auto n2v_decide = [&](double beta) {
            if (n2v_accept(V, Pv.seed(cx), Pv.wid(cx), s.hop, s.orient, beta)) {
                commit_hop();
            } else if (++s.orient >= N2V_MAX_TRIALS) {
                finish = true;  // every proposal rejected
            } else {
                bytes += 12 + 16;
                n2v_issue();
            }
        };
        // the pair-table slot of probe s.prev_w for (u, candidate z0)
        auto n2v_probe = [&]() {
            const unsigned long long key = BACK ? pair_key(z0, s.u, V.directed) : pair_key(s.u, z0, V.directed);
            const PairSlot *e = V.pt + ((pair_hash(key) + (uint64_t)(uint32_t)s.prev_w) & V.pt_mask);
            y1 = (int64_t)__ldg(&e->key);
            z2 = __ldg(&e->cnt);
            s.state = S_N2V;
        };

        switch (s.state) {
            case S_NEW: {
                int32_t L;
                int bias;
                Pv.open(s.w, cx, L, bias);
                // without the rejection states a Node2Vec walk is the
                // exponential walk (the host picks this form only then)
                if (!N2V && bias == BIAS_NODE2VEC) bias = BIAS_EXP;
                s.cap_len = L;
                s.bias = bias;
                s.len = 0;
                if (V.m == 0) {
                    finish = true;
                    break;
                }
                if (Pv.policy(cx) == TEMPEST_START_PER_NODE) {
                    z0 = __ldg(V.pn_nodes + (int64_t)(Pv.wid(cx) / (uint64_t)Pv.pn_k(cx)));
                    s.state = S_PNODE;
                    break;
                }
                const Rand4 r = walk_rand(Pv.seed(cx), Pv.wid(cx), 0u);
                const uint64_t u1 = u53_bits(r.r0, r.r1);
                s.ud = u53_bits(r.r2, r.r3);
                s.orient = ((!V.directed && (r.r3 & 1u)) ? 1u : 0u) ^ ((BACK && V.back_swap) ? 1u : 0u);
                if (Pv.policy(cx) == TEMPEST_START_UNIFORM_EDGE) {
                    int64_t k = uniform_index_k(u1, V.m);
                    if (BACK) k = V.m - 1 - k;
                    y0 = __ldg(V.st_ts + k);
                    z0 = __ldg(V.st_src + k);
                    z1 = __ldg(V.st_dst + k);
                    s.state = S_EDGE;
                } else {
                    int64_t g = sampler_index_k(u1, V.G, start_bias(bias), V.rate_start);
                    if (BACK) g = V.G - 1 - g;
                    z0 = __ldg(V.tg + g);
                    z1 = __ldg(V.tg + g + 1);
                    s.state = S_SGROUP;
                }
                break;
            }
            case S_PNODE: {
                // the walk starts at node z0 before every live edge; its
                // first hop (Philox counter 0) may take any of them
                Pv.nrow(cx)[0] = z0;
                Pv.trow(cx)[0] = INT64_MIN;
                s.len = 1;
                s.hop = 0;
                if (N2V) s.u = -1;
                s.v = z0;
                s.t = (BACK ? INT64_MAX - 1 : INT64_MIN);
                load_range(V.ngr + z0, z0, z1, z2, y0, y1, &z3);
                s.state = S_RANGE;
                break;
            }
            case S_SGROUP: {
                const int32_t x = (int32_t)((uint32_t)z0 - V.s_lo);
                const int64_t a = x > 0 ? x : 0;
                const int64_t b = (int64_t)(int32_t)((uint32_t)z1 - V.s_lo);
                const int64_t k = BACK ? b - 1 - uniform_index_k(s.ud, b - a) : a + uniform_index_k(s.ud, b - a);
                y0 = __ldg(V.st_ts + k);
                z0 = __ldg(V.st_src + k);
                z1 = __ldg(V.st_dst + k);
                s.state = S_EDGE;
                break;
            }
            case S_EDGE: {
                int32_t a = z0, b = z1;
                if (s.orient) {
                    const int32_t x = a;
                    a = b;
                    b = x;
                }
                int32_t *nrow = Pv.nrow(cx);
                int64_t *trow = Pv.trow(cx);
                nrow[0] = a;
                nrow[1] = b;
                trow[0] = INT64_MIN;
                trow[1] = y0;
                s.len = 2;
                s.hop = 1;
                if (N2V) s.u = a;
                s.v = b;
                s.t = (BACK ? y0 - 1 : y0);
                hops++;
                bytes += START_MODEL_BYTES;
                if (s.len >= s.cap_len) {
                    finish = true;
                } else {
                    load_range(V.ngr + b, z0, z1, z2, y0, y1, &z3);
                    s.state = S_RANGE;
                }
                break;
            }
            case S_RANGE: {
                // z0, z1: groups; z2: bucket base; y0, y1: first / last ts.
                // Forward, c = g0 takes every group and c = g1 none;
                // backward, the range [g0, c) flips both.
                s.g0 = z0;
                s.g1 = z1;
                if (z0 == z1) {
                    finish = true;
                } else if (s.t < y0) {
                    s.R = s.g0;  // all of the node's groups are later than t
                    if (BACK) finish = true;
                    else pick = true;
                } else if (s.t >= y1) {
                    s.R = s.g1;  // none is later than t: Gamma_t(v) is empty forward
                    if (BACK) pick = true;
                    else finish = true;
                } else if (V.bkt && s.g1 - s.g0 >= BKT_MIN_G) {
                    // y0 <= t < y1: the bucket of t brackets c
                    const int32_t *tp = V.bkt + z2 + bkt_rel(s.t, y0, z3 & 63);
                    z0 = __ldg(tp);
                    z1 = __ldg(tp + 1);
                    s.state = S_BKT;
                } else {
                    s.L = s.g0;
                    s.R = s.g1 - 1;
                    s.vL = y0;
                    s.vR = y1;
                    if (s.R - s.L == 1) {
                        pick = true;
                    } else {
                        s.prev_w = s.R - s.L;
                        const int32_t p = interp_probe(s.L, s.R, s.vL, s.vR, s.t, false);
                        z1 = p;
                        y0 = __ldg(V.ngts + p);
                        s.state = S_SEARCH;
                    }
                }
                break;
            }
            case S_BKT: {
                // c lies in [z0, z1]: groups before z0 are not later than t,
                // group z1 (or g1) is later (z0 may name an evicted group)
                z0 = max(z0, s.g0);
                if (z0 == z1) {
                    s.R = z0;
                    pick = true;
                } else {
                    s.L = z0 - 1;
                    s.R = z1;
                    s.prev_w = -1;  // bracket values unknown: bisect only
                    const int32_t p = s.L + ((s.R - s.L) >> 1);
                    z1 = p;
                    y0 = __ldg(V.ngts + p);
                    s.state = S_SEARCH;
                }
                break;
            }
            case S_SEARCH: {
                const int32_t p = z1;
                if (y0 > s.t) {
                    s.R = p;
                    s.vR = y0;
                } else {
                    s.L = p;
                    s.vL = y0;
                }
                const int32_t width = s.R - s.L;
                if (width == 1) {
                    pick = true;
                } else {
                    const bool bisect = s.prev_w < 0 || 2 * width > s.prev_w;
                    if (s.prev_w >= 0) s.prev_w = width;
                    const int32_t q = interp_probe(s.L, s.R, s.vL, s.vR, s.t, bisect);
                    z1 = q;
                    y0 = __ldg(V.ngts + q);
                }
                break;
            }
            case S_WTOT:
            case S_WSEARCH: {
                // weight-based draw: smallest k in [L, R] with gs[k + 1] <= R_w,
                // R_w = gs[c] (1 - u) (vR); y0 holds the last loaded sum
                if (s.state == S_WTOT) {
                    s.vR = __double_as_longlong(__longlong_as_double(y0) * (1.0 - (double)s.vL * 0x1.0p-53));
                } else if (__longlong_as_double(y0) <= __longlong_as_double(s.vR)) {
                    s.R = z1;
                } else {
                    s.L = z1 + 1;
                }
                if (s.L == s.R) {
                    z0 = __ldg(V.ngo + s.L);
                    z1 = __ldg(V.ngo + s.L + 1);
                    s.state = S_PICK2;
                } else {
                    const int32_t mid = s.L + ((s.R - s.L) >> 1);
                    z1 = mid;
                    y0 = __double_as_longlong(__ldg(V.gs + mid + 1));
                    s.state = S_WSEARCH;
                }
                break;
            }
            case S_PICK2: {
                const int64_t q = uniform_index_k(s.ud, (int64_t)(z1 - z0));
                const int64_t idx = BACK ? (int64_t)z1 - 1 - q : (int64_t)z0 + q;
                const Entry *e = V.ent + idx;
                y0 = __ldg(&e->ts);
                z0 = __ldg(&e->other);
                s.state = S_HOP;
                break;
            }
            case S_HOP: {
                if (!N2V) {
                    commit_hop();  // the host runs this form only where Node2Vec takes its first proposal
                } else if (s.bias != BIAS_NODE2VEC || s.u < 0) {
                    commit_hop();
                } else if (z0 == s.u) {
                    n2v_decide(V.n2v_inv_p);
                } else if (V.n2v_inv_q == 1.0) {
                    n2v_decide(1.0);  // neighbour or not, the factor is 1
                } else if (!V.pt) {
                    atomicOr(&Pv.cnt()->status, 1ull);
                    n2v_decide(V.n2v_inv_q);
                } else {
                    bytes += 32;
                    s.prev_w = 0;
                    n2v_probe();
                }
                break;
            }
            case S_N2V: {
                if (!N2V) break;  // not reached without the rejection states
                // y1: slot key, z2: its live count
                const unsigned long long key = BACK ? pair_key(z0, s.u, V.directed) : pair_key(s.u, z0, V.directed);
                if ((unsigned long long)y1 == key) {
                    n2v_decide(z2 > 0 ? 1.0 : V.n2v_inv_q);
                } else if ((unsigned long long)y1 == PAIR_EMPTY || (uint64_t)(uint32_t)s.prev_w >= V.pt_mask) {
                    n2v_decide(V.n2v_inv_q);
                } else {
                    s.prev_w++;
                    n2v_probe();
                }
                break;
            }
            default:
                break;
        }

        if (pick) {
            // c = s.R is the first group later than t; draw the next edge
            const int32_t c = s.R;
            const Rand4 r = walk_rand(Pv.seed(cx), Pv.wid(cx), s.hop);
            const uint64_t u1 = u53_bits(r.r0, r.r1);
            const int hb = hop_bias(V, s.bias, Pv.cnt());
            s.state = S_PICK2;
            if (N2V && hb == BIAS_NODE2VEC) {
                s.orient = 0;  // proposal 0 is the exponential draw of this hop's block
                n2v_issue();
            } else if (BACK) {
                // groups [g0, c) in the mirrored order (latest first)
                if (hb == BIAS_UNIFORM) {
                    s.ud = u1;
                    z0 = __ldg(V.ngo + s.g0);
                    z1 = __ldg(V.ngo + c);
                } else {
                    s.ud = u53_bits(r.r2, r.r3);
                    const int32_t gg =
                        c - 1 - (int32_t)sampler_index_k(u1, (int64_t)(c - s.g0), start_bias(hb), V.rate_hop);
                    z0 = __ldg(V.ngo + gg);
                    z1 = __ldg(V.ngo + gg + 1);
                }
            } else if (hb == BIAS_UNIFORM) {
                s.ud = u1;
                z0 = __ldg(V.ngo + c);
                z1 = __ldg(V.ngo + s.g1);
            } else if (hb == BIAS_EXP_WEIGHT) {
                // weight of Gamma first, then a bisection on the suffix sums
                s.ud = u53_bits(r.r2, r.r3);
                s.vL = (int64_t)u1;
                s.L = c;
                s.R = s.g1 - 1;
                y0 = __double_as_longlong(__ldg(V.gs + c));
                s.state = S_WTOT;
            } else {
                s.ud = u53_bits(r.r2, r.r3);
                const int64_t j = sampler_index_k(u1, (int64_t)(s.g1 - c), hb, V.rate_hop);
                z0 = __ldg(V.ngo + c + j);
                z1 = __ldg(V.ngo + c + j + 1);
            }
        }
        // rows of the walks that ended here: the whole warp writes their
        // padding (node -1, ts INT64_MIN up to the row end), 32 consecutive
        // cells per store, while the row's head is still in L2
        unsigned fin = __ballot_sync(0xffffffffu, finish);
        if (fin) {
            unsigned long long my_n = 0, my_t = 0;
            int32_t my_len = 0, my_cap = 0;
            if (finish) {
                Pv.finish(cx, s.len);
                my_n = (unsigned long long)Pv.nrow(cx);
                my_t = (unsigned long long)Pv.trow(cx);
                my_len = s.len;
                my_cap = Pv.cap(cx);
                s.state = S_FETCH;
            }
            while (fin) {
                const int src = __ffs(fin) - 1;
                fin &= fin - 1;
                int32_t *nr = reinterpret_cast<int32_t *>(__shfl_sync(0xffffffffu, my_n, src));
                int64_t *tr = reinterpret_cast<int64_t *>(__shfl_sync(0xffffffffu, my_t, src));
                const int32_t l = __shfl_sync(0xffffffffu, my_len, src);
                const int32_t cp = __shfl_sync(0xffffffffu, my_cap, src);
                for (int32_t i = l + lane; i < cp; i += 32) {
                    __stcs(nr + i, -1);  // streaming stores: padding is not read back
                    __stcs(reinterpret_cast<long long *>(tr) + i, (long long)INT64_MIN);
                }
            }
        }
    }
    hops = warp_sum(hops);
    bytes = warp_sum(bytes);
    if (lane == 0 && hops) {
        atomicAdd(&Pv.cnt()->hops, hops);
        atomicAdd(&Pv.cnt()->model_bytes, bytes);
    }
}

// ---------------------------------------------------------------------------
// Lane walker (TEMPEST_SCHED_LANE): persistent like the streaming walker, but
// every iteration advances each lane by one whole hop (or one start) in
// straight-line code, so the lanes of a warp run the same instructions
// together (the hop-synchronous kernels' efficiency) while a lane whose walk
// ends takes the next walk id at once (no waiting for the warp's longest
// walk).  The hop's dependent loads (node record, bucket pair, search probes,
// group offsets, entry) are issued in sequence; occupancy hides them.
// ---------------------------------------------------------------------------

// First group of [g0, g1) later than t, for tlo <= t < thi (the node's first
// and last group timestamps): through the time buckets of a big node, else by
// interpolation on the group timestamps with a bisection fallback.
__device__ __forceinline__ int32_t lane_first_later(const WalkView &V, int32_t g0, int32_t g1, int32_t tb, int32_t bs,
                                                    int64_t tlo, int64_t thi, int64_t t)
{
    if (V.bkt && g1 - g0 >= BKT_MIN_G) {
        const int32_t k = bkt_rel(t, tlo, bs & 63);
        return upper_bound_ts(V.ngts, max(__ldg(V.bkt + tb + k), g0), __ldg(V.bkt + tb + k + 1), t);
    }
    // ngts[L] <= t < ngts[R]
    int32_t L = g0, R = g1 - 1;
    int64_t vL = tlo, vR = thi;
    int32_t prev_w = R - L;
    bool bisect = false;  // interpolate first; bisect after a probe that did not halve the bracket
    while (R - L > 1) {
        const int32_t p = interp_probe(L, R, vL, vR, t, bisect);
        const int64_t a = __ldg(V.ngts + p);
        if (a > t) {
            R = p;
            vR = a;
        } else {
            L = p;
            vL = a;
        }
        bisect = 2 * (R - L) > prev_w;
        prev_w = R - L;
    }
    return R;
}

// The seed and counters a draw helper needs, per request.
struct DrawCtx {
    uint64_t seed;
    WalkCounters *cnt;
};

// With PAD, the first LANE_STAGE cells of each walk wait in shared memory
// (LANE_STAGE + 1 words per lane, so that lanes writing their own cells and
// the warp reading one lane's cells both stay off shared bank conflicts);
// when the walk ends, the warp writes the row in one pass, cells and padding
// together, so each 32-byte sector of the row is written whole by one store
// instruction instead of once by scattered cell stores and again by the
// padding (two partial writes of the same sector, merged in DRAM when L2
// has evicted the first).  Cells past the staged ones go to the row directly.
constexpr int LANE_STAGE = 8;
constexpr int LANE_STAGE_STRIDE = LANE_STAGE + 1;

template <class P, int MINB, bool N2V, bool BACK, bool PAD>
__global__ void __launch_bounds__(256, MINB) k_walks_lane(const WalkView V, const P Pv, unsigned long long *next_walk)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    __shared__ int32_t s_node[PAD ? 256 * LANE_STAGE_STRIDE : 1];
    __shared__ long long s_ts[PAD ? 256 * LANE_STAGE_STRIDE : 1];
    const int my_stage = PAD ? (int)threadIdx.x * LANE_STAGE_STRIDE : 0;
    // cell i of the lane's walk: staged (PAD, i < LANE_STAGE) or to its row
    auto put = [&](const typename P::Ctx &c, int32_t i, int32_t nv, int64_t tv) {
        if (PAD && i < LANE_STAGE) {
            s_node[my_stage + i] = nv;
            s_ts[my_stage + i] = (long long)tv;
        } else {
            Pv.nrow(c)[i] = nv;
            Pv.trow(c)[i] = tv;
        }
    };
    typename P::Ctx cx;
    int64_t w = 0;
    int32_t v = 0, u = -1, len = 0, cap_len = 0, bias = 0;
    int64_t t = 0;
    int mode = 0;  // 0: needs a walk, 1: fresh walk, 2: walking, 3: no more walks
    unsigned long long hops = 0, bytes = 0;
    const int64_t N = Pv.total();
    constexpr int64_t WALK_CHUNK = 256;
    int64_t q_next = 0, q_end = 0;
    while (true) {
        unsigned need = __ballot_sync(0xffffffffu, mode == 0);
        while (need) {
            if (q_next >= q_end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(next_walk, (unsigned long long)WALK_CHUNK);
                base = __shfl_sync(0xffffffffu, base, 0);
                if ((int64_t)base >= N) {
                    if (mode == 0) mode = 3;
                    break;
                }
                q_next = (int64_t)base;
                q_end = min(N, q_next + WALK_CHUNK);
            }
            const int64_t avail = q_end - q_next;
            const int rank = __popc(need & lt);
            const int take = (int)min((int64_t)__popc(need), avail);
            if (mode == 0 && rank < take) {
                w = q_next + rank;
                mode = 1;
            }
            q_next += take;
            need = __ballot_sync(0xffffffffu, mode == 0);
        }
        if (__all_sync(0xffffffffu, mode == 3)) break;

        bool finish = false;
        if (mode == 1) {
            int32_t L;
            int b;
            Pv.open(w, cx, L, b);
            if (!N2V && b == BIAS_NODE2VEC) b = BIAS_EXP;  // launched only when that is exact (p = q = 1)
            cap_len = L;
            bias = b;
            mode = 2;
            if (V.m == 0) {
                len = 0;
                finish = true;
            } else if (Pv.policy(cx) == TEMPEST_START_PER_NODE) {
                v = __ldg(V.pn_nodes + (int64_t)(Pv.wid(cx) / (uint64_t)Pv.pn_k(cx)));
                put(cx, 0, v, INT64_MIN);
                len = 1;
                u = -1;
                t = BACK ? INT64_MAX - 1 : INT64_MIN;
            } else {
                const Rand4 r = walk_rand(Pv.seed(cx), Pv.wid(cx), 0u);
                const uint64_t k1 = u53_bits(r.r0, r.r1), k2 = u53_bits(r.r2, r.r3);
                int64_t k;
                if (Pv.policy(cx) == TEMPEST_START_UNIFORM_EDGE) {
                    k = uniform_index_k(k1, V.m);
                    if (BACK) k = V.m - 1 - k;
                } else {
                    int64_t g = sampler_index_k(k1, V.G, start_bias(bias), V.rate_start);
                    if (BACK) g = V.G - 1 - g;
                    int64_t a, e;
                    ts_group_range(V, g, a, e);
                    k = BACK ? e - 1 - uniform_index_k(k2, e - a) : a + uniform_index_k(k2, e - a);
                }
                int32_t s0 = __ldg(V.st_src + k), d0 = __ldg(V.st_dst + k);
                const int64_t t0 = __ldg(V.st_ts + k);
                if ((((!V.directed && (r.r3 & 1u)) ? 1u : 0u) ^ ((BACK && V.back_swap) ? 1u : 0u)) != 0u) {
                    const int32_t x = s0;
                    s0 = d0;
                    d0 = x;
                }
                put(cx, 0, s0, INT64_MIN);
                put(cx, 1, d0, t0);
                len = 2;
                u = s0;
                v = d0;
                t = BACK ? t0 - 1 : t0;
                hops++;
                bytes += START_MODEL_BYTES;
                if (len >= cap_len) finish = true;
            }
        } else if (mode == 2) {
            // one hop from v at search time t
            const uint32_t hop = (uint32_t)(len - 1);
            int32_t g0, g1, tb, bs;
            int64_t tlo, thi;
            load_range(V.ngr + v, g0, g1, tb, tlo, thi, &bs);
            int32_t c = g0;
            if (g0 == g1) {
                finish = true;
            } else if (t < tlo) {
                c = g0;
            } else if (t >= thi) {
                c = g1;
            } else {
                c = lane_first_later(V, g0, g1, tb, bs, tlo, thi, t);
            }
            if (!finish && (BACK ? c == g0 : c == g1)) finish = true;  // Gamma_t(v) is empty
            if (!finish) {
                const DrawCtx D{Pv.seed(cx), Pv.cnt()};
                const uint64_t wid = Pv.wid(cx);
                Entry e;
                bool ok = true;
                if (N2V && bias == BIAS_NODE2VEC) {
                    ok = draw_n2v(V, D, (int64_t)wid, hop, g0, c, g1, u, e, bytes);
                } else if (BACK) {
                    e = draw_entry_back(V, D, (int64_t)wid, hop, bias, g0, c);
                } else {
                    e = draw_entry(V, D, (int64_t)wid, hop, bias, c, g1);
                }
                if (!ok) {
                    finish = true;  // every Node2Vec proposal rejected
                } else {
                    put(cx, len, e.other, e.ts);
                    hops++;
                    bytes += hop_model_bytes((int64_t)(g1 - g0));
                    len++;
                    u = v;
                    v = e.other;
                    t = BACK ? e.ts - 1 : e.ts;
                    if (len >= cap_len) finish = true;
                }
            }
        }
        // rows of the walks that ended here: the whole warp writes each row,
        // its staged cells and its padding, 32 consecutive cells per
        // streaming store (PAD; else one pass after the launch pads every
        // row)
        unsigned fin = __ballot_sync(0xffffffffu, finish);
        if (!PAD) {
            if (finish) {
                Pv.finish(cx, len);
                mode = 0;
            }
        } else if (fin) {  // every lane of the warp takes part in the padding loop
            unsigned long long my_n = 0, my_t = 0;
            int32_t my_len = 0, my_cap = 0;
            if (finish) {
                Pv.finish(cx, len);
                my_n = (unsigned long long)Pv.nrow(cx);
                my_t = (unsigned long long)Pv.trow(cx);
                my_len = len;
                my_cap = Pv.cap(cx);
                mode = 0;
            }
            __syncwarp();  // the staged cells of every lane are visible to the warp
            const int warp_stage = (int)(threadIdx.x & ~31u) * LANE_STAGE_STRIDE;
            while (fin) {
                const int src = __ffs(fin) - 1;
                fin &= fin - 1;
                int32_t *nr = reinterpret_cast<int32_t *>(__shfl_sync(0xffffffffu, my_n, src));
                int64_t *tr = reinterpret_cast<int64_t *>(__shfl_sync(0xffffffffu, my_t, src));
                const int32_t l = __shfl_sync(0xffffffffu, my_len, src);
                const int32_t cp = __shfl_sync(0xffffffffu, my_cap, src);
                const int sb = warp_stage + src * LANE_STAGE_STRIDE;
                for (int32_t i = lane; i < cp; i += 32) {
                    if (i >= LANE_STAGE && i < l) continue;  // written at its hop
                    int32_t nv = -1;
                    long long tv = (long long)INT64_MIN;
                    if (i < l) {
                        nv = s_node[sb + i];
                        tv = s_ts[sb + i];
                    }
                    __stcs(nr + i, nv);
                    __stcs(reinterpret_cast<long long *>(tr) + i, tv);
                }
            }
            __syncwarp();  // a lane's next walk stages its cells after these reads
        }
    }
    hops = warp_sum(hops);
    bytes = warp_sum(bytes);
    if (lane == 0 && hops) {
        atomicAdd(&Pv.cnt()->hops, hops);
        atomicAdd(&Pv.cnt()->model_bytes, bytes);
    }
}

// Padding of every row after its walk: node -1, ts INT64_MIN from len to the
// row end.  A warp takes 32 consecutive rows per step: one coalesced load of
// their lengths, then row by row with the lanes on consecutive cells.
__global__ void __launch_bounds__(256) k_pad_rows(int64_t n_walks, int32_t cap, const int32_t *__restrict__ len,
                                                  int32_t *node, int64_t *ts)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; w0 < n_walks; w0 += warps * 32) {
        const int64_t w = w0 + lane;
        warp_pad_walk_rows(node, ts, cap, w < n_walks ? w : -1, w < n_walks ? len[w] : cap, lane);
    }
}

void pad_rows(tempest_t *h, int64_t n, int32_t cap, const int32_t *len, int32_t *node, int64_t *ts)
{
    int64_t pgrid = (n + 7) / 8;
    const int64_t pcap = (int64_t)h->num_sms * 16;
    if (pgrid > pcap) pgrid = pcap;
    if (n > 0) k_pad_rows<<<(unsigned)pgrid, 256, 0, h->stream>>>(n, cap, len, node, ts);
}

// Launches the streaming walker with the register budget the CTAs-per-SM
// knob asks for (0: the 64-register build at its occupancy limit).
// n2v: a walk of the launch may take Node2Vec hops with p, q not both 1
template <class P, bool BACK>
static void launch_stream_dir(tempest_t *h, const WalkView &V, const P &Pv, unsigned long long *next, int64_t total,
                              cudaStream_t st, bool n2v)
{
    static int occ4 = 0, occ5 = 0, occn = 0;
    if (occ4 == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ4, k_walks_stream<P, 4, false, BACK>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ5, k_walks_stream<P, 5, false, BACK>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occn, k_walks_stream<P, 3, true, BACK>, 256, 0);
        if (occ4 < 1) occ4 = 1;
        if (occ5 < 1) occ5 = 1;
        if (occn < 1) occn = 1;
    }
    const bool wide = h->stream_ctas > 4 && !n2v;
    const int occ = n2v ? occn : (wide ? occ5 : occ4);
    const int bps = h->stream_ctas > 0 ? std::min(h->stream_ctas, occ) : occ;
    int64_t grid = (int64_t)h->num_sms * bps;
    const int64_t need = (total + 255) / 256;
    if (grid > need) grid = need;
    if (n2v) k_walks_stream<P, 3, true, BACK><<<(unsigned)grid, 256, 0, st>>>(V, Pv, next);
    else if (wide) k_walks_stream<P, 5, false, BACK><<<(unsigned)grid, 256, 0, st>>>(V, Pv, next);
    else k_walks_stream<P, 4, false, BACK><<<(unsigned)grid, 256, 0, st>>>(V, Pv, next);
}

// CTAs per SM the Node2Vec lane walker is built for: one request's walks fit
// 64 registers without spills, the multi-request form needs more.
template <class P>
constexpr int LANE_N2V_MINB = std::is_same<P, OneReq>::value ? 4 : 3;

template <class P, bool BACK, bool PAD>
static void launch_lane_pad(tempest_t *h, const WalkView &V, const P &Pv, unsigned long long *next, int64_t total,
                            cudaStream_t st, bool n2v)
{
    static int occ = 0, occ5 = 0, occ6 = 0, occn = 0;
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_walks_lane<P, 4, false, BACK, PAD>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ5, k_walks_lane<P, 5, false, BACK, PAD>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ6, k_walks_lane<P, 6, false, BACK, PAD>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occn, k_walks_lane<P, LANE_N2V_MINB<P>, true, BACK, PAD>, 256, 0);
        if (occ < 1) occ = 1;
        if (occ5 < 1) occ5 = 1;
        if (occ6 < 1) occ6 = 1;
        if (occn < 1) occn = 1;
    }
    // the build for the CTAs per SM the knob asks for: 4 (no spills), 5 or
    // 6 (fewer registers, more warps to hide the hops' dependent loads)
    const int minb = n2v ? 0 : (h->stream_ctas >= 6 ? 6 : (h->stream_ctas == 5 ? 5 : 4));
    const int o = n2v ? occn : (minb == 6 ? occ6 : (minb == 5 ? occ5 : occ));
    const int bps = h->stream_ctas > 0 ? std::min(h->stream_ctas, o) : o;
    int64_t grid = (int64_t)h->num_sms * bps;
    const int64_t need = (total + 255) / 256;
    if (grid > need) grid = need;
    if (n2v) k_walks_lane<P, LANE_N2V_MINB<P>, true, BACK, PAD><<<(unsigned)grid, 256, 0, st>>>(V, Pv, next);
    else if (minb == 6) k_walks_lane<P, 6, false, BACK, PAD><<<(unsigned)grid, 256, 0, st>>>(V, Pv, next);
    else if (minb == 5) k_walks_lane<P, 5, false, BACK, PAD><<<(unsigned)grid, 256, 0, st>>>(V, Pv, next);
    else k_walks_lane<P, 4, false, BACK, PAD><<<(unsigned)grid, 256, 0, st>>>(V, Pv, next);
}

template <class P, bool BACK>
static void launch_lane_dir(tempest_t *h, const WalkView &V, const P &Pv, unsigned long long *next, int64_t total,
                            cudaStream_t st, bool n2v, bool pad)
{
    if (pad) launch_lane_pad<P, BACK, true>(h, V, Pv, next, total, st, n2v);
    else launch_lane_pad<P, BACK, false>(h, V, Pv, next, total, st, n2v);
}

// The persistent walker of the handle's form (the lane walker for
// TEMPEST_SCHED_LANE, else the streaming walker).
template <class P>
static void launch_stream(tempest_t *h, const WalkView &V, const P &Pv, unsigned long long *next, int64_t total,
                          cudaStream_t st, bool n2v, bool pad = true)
{
    if (h->sched == TEMPEST_SCHED_LANE) {
        if (V.back) launch_lane_dir<P, true>(h, V, Pv, next, total, st, n2v, pad);
        else launch_lane_dir<P, false>(h, V, Pv, next, total, st, n2v, pad);
        return;
    }
    if (V.back) launch_stream_dir<P, true>(h, V, Pv, next, total, st, n2v);
    else launch_stream_dir<P, false>(h, V, Pv, next, total, st, n2v);
}

// Events bracketing the walk kernels of a call (created on first use).
static void kernel_mark(tempest_t *h, int which)
{
    if (!h->kev[which]) cudaEventCreate(&h->kev[which]);
    cudaEventRecord(h->kev[which], h->stream);
    if (which == 1) h->kev_valid = true;
}

int walks_multi_launch(tempest_t *h, int direction, const ReqDesc *dev_reqs, int n_req, int64_t total,
                       WalkCounters *cnt, cudaStream_t st, bool clear, bool may_n2v)
{
    // the walk-id counter always restarts; the statistics only when asked
    if (clear) cudaMemsetAsync(cnt, 0, sizeof(WalkCounters), st);
    else cudaMemsetAsync(&cnt->pad, 0, sizeof(cnt->pad), st);
    if (total <= 0 || n_req <= 0) return cuda_check(h, cudaGetLastError(), "walks multi");
    tempest_t *vh = view_handle(h, direction);
    if (!vh) return fail(h, TEMPEST_EINVAL, "backward walks of a directed graph need tempest_enable_backward");
    WalkView V = make_view(vh, direction);
    view_n2v(V, h);  // the pair table and parameters live on the main handle
    const bool mark = st == h->stream;
    if (mark) kernel_mark(h, 0);
    const bool n2v = may_n2v && (V.n2v_inv_p != 1.0 || V.n2v_inv_q != 1.0);
    launch_stream(h, V, ManyReq{dev_reqs, n_req, total, cnt}, &cnt->pad, total, st, n2v);
    if (mark) kernel_mark(h, 1);
    return cuda_check(h, cudaGetLastError(), "walks multi");
}

__global__ void k_sample_index(const uint64_t *__restrict__ ub, const int64_t *__restrict__ n, int64_t count,
                               int bias, ExpRate R, int64_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ub[i] & ((1ull << 53) - 1ull);
        const int64_t m = n[i];
        out[i] = m >= 1 ? sampler_index_k(k, m, bias, R) : 0;
    }
}

int sample_index_run(tempest_t *h, const uint64_t *ub, const int64_t *n, int64_t count, int bias, double lambda,
                     int64_t *out)
{
    if (count <= 0) return TEMPEST_OK;
    const ExpRate R{lambda, (float)lambda, (float)(1.0 / lambda)};
    int64_t grid = (count + 255) / 256;
    const int64_t cap = (int64_t)h->num_sms * 16;
    if (grid > cap) grid = cap;
    k_sample_index<<<(unsigned)grid, 256, 0, h->stream>>>(ub, n, count, bias, R, out);
    return cuda_check(h, cudaGetLastError(), "sample_index");
}

tempest_t *view_handle(tempest_t *h, int direction)
{
    if (direction == 0 || !h->directed) return h;
    tempest_t *r = h->rev;
    if (!r) return nullptr;
    // the reversed index follows the main handle's stream and settings
    r->stream = h->stream;
    r->lam_hop = h->lam_hop;
    r->lam_start = h->lam_start;
    if (r->bkt_log != h->bkt_log) {
        r->bkt_log = h->bkt_log;
        r->bkt_ver = -1;
    }
    return r;
}

WalkView make_view(tempest_t *h, int back)
{
    WalkView V;
    V.back = back;
    V.back_swap = back && !h->directed;
    V.st_src = h->st_src[h->cur].as<int32_t>() + h->s_lo;
    V.st_dst = h->st_dst[h->cur].as<int32_t>() + h->s_lo;
    V.st_ts = h->st_ts[h->cur].as<int64_t>() + h->s_lo;
    V.m = h->m;
    V.tg = h->tg.as<int32_t>() + h->tg_lo;
    V.s_lo = (uint32_t)(uint64_t)(h->s_base + h->s_lo);
    V.G = h->G;
    V.ngr = h->ngr.as<NodeRange>();
    V.ngo = h->ngo.as<int32_t>();
    V.ngts = h->ngts.as<int64_t>();
    V.ent = h->ent.as<Entry>();
    const bool bk = h->n_big > 0 && h->bkt_ver == h->state_ver;
    V.bkt = bk ? h->bkt.as<int32_t>() : nullptr;
    V.pn_nodes = h->pn_ver == h->state_ver ? h->pn_nodes.as<int32_t>() : nullptr;
    V.gs = !back && h->w_on && h->w_valid && h->w_ver == h->state_ver ? h->gs.as<double>() : nullptr;
    V.bkt_log = h->bkt_log;
    V.directed = h->directed;
    const double ls = h->lam_start > 0.0 ? h->lam_start : (h->G > 0 ? 1.0 / (double)h->G : 1.0);
    V.rate_hop = ExpRate{h->lam_hop, (float)h->lam_hop, (float)(1.0 / h->lam_hop)};
    V.rate_start = ExpRate{ls, (float)ls, (float)(1.0 / ls)};
    view_n2v(V, h);
    return V;
}

void view_n2v(WalkView &V, const tempest_t *h)
{
    V.pt = h->pt_on ? h->pt.as<PairSlot>() : nullptr;
    V.pt_mask = h->pt_on ? (uint64_t)h->pt_cap - 1 : 0;
    V.n2v_inv_p = 1.0 / h->n2v_p;
    V.n2v_inv_q = 1.0 / h->n2v_q;
    V.n2v_bmax = std::max(std::max(V.n2v_inv_p, 1.0), V.n2v_inv_q);
}

int walks_run(tempest_t *h, const WalkRequest &rq)
{
    int rc;
    h->kev_valid = false;
    tempest_t *vh = view_handle(h, rq.direction);
    if (!vh) return fail(h, TEMPEST_EINVAL, "backward walks of a directed graph need tempest_enable_backward");
    NvtxStages stage;
    stage.next("walks: index");
    if ((rc = prepare_walk_index(vh))) return rc;
    if (rq.direction == 0 &&
        ((!rq.bias_arr && rq.bias == TEMPEST_BIAS_EXP_WEIGHT) || rq.want_w || (rq.bias_arr && h->w_on)))
        if ((rc = prepare_weights(h))) return rc;
    if ((rc = ensure(h, h->wcnt, sizeof(WalkCounters)))) return rc;
    cudaStream_t st = h->stream;
    cudaMemsetAsync(h->wcnt.p, 0, sizeof(WalkCounters), st);
    WalkView V = make_view(vh, rq.direction);
    view_n2v(V, h);  // the pair table and parameters live on the main handle
    WalkOut O;
    O.n_walks = rq.n_walks;
    O.cap = rq.cap;
    O.max_len = rq.max_len;
    O.len_arr = rq.len_arr;
    O.bias = rq.bias;
    O.bias_arr = rq.bias_arr;
    O.start_policy = rq.start_policy;
    O.pn_k = rq.pn_k;
    O.seed = rq.seed;
    O.node = rq.node;
    O.ts = rq.ts;
    O.len = rq.len;
    O.cnt = h->wcnt.as<WalkCounters>();
    int64_t launches = 0;
    for (int t = 0; t < 5; t++) h->coop_tier_launches[t] = 0;
    stage.next("walks: kernels");
    if (rq.n_walks > 0) {
        if (h->sched == TEMPEST_SCHED_COOP || h->sched == TEMPEST_SCHED_GRAPH) {
            kernel_mark(h, 0);
            int rc2 = h->sched == TEMPEST_SCHED_COOP ? coop_run(h, V, O, launches) : graph_run(h, V, O, launches);
            if (rc2) return rc2;
            kernel_mark(h, 1);
            // one streaming pass pads the rows (padding inside the short
            // hop-synchronous kernels measured slower than this pass)
            int64_t pgrid = (rq.n_walks + 7) / 8;
            const int64_t pcap = (int64_t)h->num_sms * 16;
            if (pgrid > pcap) pgrid = pcap;
            k_pad_rows<<<(unsigned)pgrid, 256, 0, st>>>(rq.n_walks, rq.cap, rq.len, rq.node, rq.ts);
            launches++;
        } else if (h->sched == TEMPEST_SCHED_FULL_WALK) {
            int64_t grid = (rq.n_walks + 255) / 256;
            const int64_t cap = (int64_t)h->num_sms * 8;
            if (grid > cap) grid = cap;
            kernel_mark(h, 0);
            k_walks_full<<<(unsigned)grid, 256, 0, st>>>(V, O);
            kernel_mark(h, 1);
            launches++;
        } else {
            kernel_mark(h, 0);
            const bool n2v = (rq.bias_arr ? rq.may_n2v != 0 : rq.bias == TEMPEST_BIAS_NODE2VEC) &&
                             (V.n2v_inv_p != 1.0 || V.n2v_inv_q != 1.0);
            // the lane walker pads rows as walks end, or leaves it to one pass
            const bool sep = h->sched == TEMPEST_SCHED_LANE && h->pad_pass && !rq.no_pad;
            launch_stream(h, V, OneReq{O}, &O.cnt->pad, rq.n_walks, st, n2v, !sep && !rq.no_pad);
            if (sep) {
                int64_t pgrid = (rq.n_walks + 7) / 8;
                const int64_t pcap = (int64_t)h->num_sms * 16;
                if (pgrid > pcap) pgrid = pcap;
                k_pad_rows<<<(unsigned)pgrid, 256, 0, st>>>(rq.n_walks, rq.cap, rq.len, rq.node, rq.ts);
                launches++;
            }
            kernel_mark(h, 1);
            launches += 1;
        }
    }
    h->last_ws.n_walks = rq.n_walks;
    h->last_ws.launches = launches;
    for (int t = 0; t < 5; t++) h->last_ws.tier_launches[t] = h->coop_tier_launches[t];
    return cuda_check(h, cudaGetLastError(), "walk launch");
}

}  // namespace tw
