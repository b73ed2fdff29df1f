// nodeview.cu -- the node-and-timestamp-grouped view of Tempest Sec. 2.3,
// kept up to date under the sliding window of Sec. 2.6 with work that grows
// with the batch, not with the window.
//
// Layout ("slack" layout).  Every node with entries owns a region of the
// entry pool (16-byte Entry records) and a region of the group pools (int32
// group start, int64 group timestamp).  Its live entries are [e_lo, e_hi) in
// (ts, arrival) order, its live groups [g_lo, g_hi); group g's entries start
// at ngo[g] and the slot after the last live group holds e_hi, so every
// group's range is [ngo[g], ngo[g + 1]).  Each region has room to grow
// (capacity x + (x >> shift) + 16 for x live items).
//
// Per appended batch (the batch starts no earlier than the store ends):
//   1. evicted entries are counted per node (the evicted edges are a store
//      prefix, so every node loses a prefix of its entries); each such node
//      advances e_lo, finds its first kept group by binary search and clamps
//      that group's start;
//   2. the batch's entries are sorted by node (stable radix sort; the batch
//      is in (ts, arrival) order so each node's entries stay in that order);
//      one compaction numbers the node runs and the new groups (a batch
//      entry opens a group unless it has the timestamp of the entry before it
//      in its node, or of the node's last group);
//   3. one thread per run appends in place when the node's regions have room,
//      otherwise takes fresh regions from the pools' bump pointers and queues
//      a move of the node's live entries and groups;
//   4. the moves run as chunked copies (group starts rebased), then the batch
//      entries, new groups and each node's closing group slot are scattered
//      into place.  A node whose regions have no room at the end but whose
//      evicted front can hold its live items moves back to the front of its
//      own regions (a sliding window's steady state), otherwise it takes fresh
//      regions from the pools.
// Nothing reads or writes the parts of the view the batch does not touch.  A
// pool that runs out, a batch that merges into the middle of the store, or
// the first batch rebuild the whole view from the store (the same compaction
// over a radix sort of all entries), leaving every region with slack.
#include "engine.cuh"
#include "prims.cuh"
#include "sortscan.cuh"

namespace tw {

namespace {

constexpr int RELOC_CHUNK = 1024;

// Capacity of a region for x items: slack x >> shift, and half as much again
// for a node of at least big_min entries (a hub slides back to the front of
// its regions once its live range reaches their end; more slack makes that
// rarer, and the copy ahead of it spans fewer of the batches).
__device__ __forceinline__ int64_t region_cap(int64_t x, int shift, bool big)
{
    return x + (x >> shift) + (big ? (x >> (shift + 1)) : 0) + 16;
}

// The entry of store item i (directed: edge i under its source; undirected:
// item 2p under src_p, item 2p + 1 under dst_p).
struct Items {
    const int32_t *src, *dst;
    const int64_t *ts;
    int directed;
    __device__ __forceinline__ int64_t edge(int64_t i) const { return directed ? i : (i >> 1); }
    __device__ __forceinline__ bool side(int64_t i) const { return !directed && (i & 1); }
    __device__ __forceinline__ uint32_t key(int64_t i) const
    {
        const int64_t e = edge(i);
        return (uint32_t)(side(i) ? dst[e] : src[e]);
    }
    __device__ __forceinline__ uint32_t val(int64_t i) const { return (uint32_t)i; }
    __device__ __forceinline__ Entry entry(int64_t i, uint32_t slot_base) const
    {
        const int64_t e = edge(i);
        Entry x;
        x.ts = ts[e];
        x.other = side(i) ? src[e] : dst[e];
        x.slot = (int32_t)(slot_base + (uint32_t)i);
        return x;
    }
};

// ---------------------------------------------------------------- full build

__global__ void k_nv_entries(const uint32_t *__restrict__ vb, Items it, int64_t M, uint32_t slot_base, Entry *E)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x)
        E[p] = it.entry(vb[p], slot_base);
}

// An appending batch's entries in sorted order (kb: batch-local node ids,
// vb: batch items), packed, with a byte per entry for the run scan: bit 0 a
// node run starts here, bit 1 a (node, timestamp) group starts here (against
// the previous entry of the run, or at a run start against the node's last
// live group before the batch).  The previous entry's id and timestamp come
// from the lane before (lane 0 loads them), so the scan passes read one byte
// per entry instead of the entries.
__global__ void __launch_bounds__(256) k_nv_entries_runs(const uint32_t *__restrict__ vb,
                                                         const uint32_t *__restrict__ kb, Items it, int64_t M,
                                                         uint32_t slot_base, const int32_t *__restrict__ touched,
                                                         const NodeRange *__restrict__ ngr, Entry *E, uint8_t *flags)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count: every lane of a warp takes part in the shuffles
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; base < M; base += stride) {
        const int64_t p = base + lane;
        const bool ok = p < M;
        Entry x{};
        uint32_t k = 0;
        if (ok) {
            x = it.entry(vb[p], slot_base);
            k = kb[p];
            E[p] = x;
        }
        uint32_t kprev = __shfl_up_sync(0xffffffffu, k, 1);
        long long tprev = __shfl_up_sync(0xffffffffu, (long long)x.ts, 1);
        if (lane == 0 && ok && p > 0) {
            kprev = kb[p - 1];
            tprev = it.entry(vb[p - 1], slot_base).ts;
        }
        if (ok) {
            const bool nc = p == 0 || k != kprev;
            bool gc;
            if (nc) {
                const NodeRange g = ngr[touched[k]];
                gc = g.g_lo == g.g_hi || g.t_last != x.ts;
            } else {
                gc = tprev != x.ts;
            }
            flags[p] = (uint8_t)((nc ? 1 : 0) | (gc ? 2 : 0));
        }
    }
}

// Node runs and groups over all entries in (node, ts, arrival) order.
struct BuildRunOp {
    const uint32_t *kb;
    const Entry *E;
    int32_t *run_of, *fx, *run_node, *run_pos, *run_g;
    __device__ __forceinline__ uint64_t value(int64_t p) const
    {
        const bool nc = p == 0 || kb[p] != kb[p - 1];
        const bool gc = nc || E[p].ts != E[p - 1].ts;
        return ((uint64_t)nc << 32) | (uint64_t)gc;
    }
    __device__ __forceinline__ void emit(int64_t p, uint64_t v, uint64_t ex) const
    {
        const uint32_t r = (uint32_t)(ex >> 32) + (uint32_t)(v >> 32) - 1u;
        run_of[p] = (int32_t)r;
        fx[p] = (int32_t)(uint32_t)ex;
        if (v >> 32) {
            run_node[r] = (int32_t)kb[p];
            run_pos[r] = (int32_t)p;
            run_g[r] = (int32_t)(uint32_t)ex;
        }
    }
};

// Region sizes of each run: low 32 bits entries, high 32 bits groups (+1
// for the slot after the last group).
struct CapOp {
    const int32_t *run_pos, *run_g;
    int shift;
    int32_t big_min;
    int32_t *run_de, *run_dg;
    __device__ __forceinline__ uint64_t value(int64_t r) const
    {
        const int64_t c = run_pos[r + 1] - run_pos[r], gc = run_g[r + 1] - run_g[r];
        const bool big = c >= big_min;
        return ((uint64_t)(region_cap(gc, shift, big) + 1) << 32) | (uint64_t)region_cap(c, shift, big);
    }
    __device__ __forceinline__ void emit(int64_t r, uint64_t, uint64_t ex) const
    {
        run_de[r] = (int32_t)(uint32_t)ex;
        run_dg[r] = (int32_t)(uint32_t)(ex >> 32);
    }
};

__global__ void k_nv_tail(int32_t *run_pos, int32_t *run_g, int32_t *fx, const uint64_t *tot, int64_t n)
{
    const uint64_t t = *tot;
    const int64_t R = (int64_t)(t >> 32);
    run_pos[R] = (int32_t)n;
    run_g[R] = (int32_t)(uint32_t)t;
    if (fx) fx[n] = (int32_t)(uint32_t)t;
}

__global__ void k_nv_build_nodes(const int32_t *__restrict__ run_node, const int32_t *__restrict__ run_pos,
                                 const int32_t *__restrict__ run_g, const int32_t *__restrict__ run_de,
                                 const int32_t *__restrict__ run_dg, const Entry *__restrict__ E, int64_t S,
                                 int shift, int32_t big_min, int4 *nrec, NodeRange *ngr, int2 *nbeg, int32_t *ngo,
                                 int32_t *act)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < S; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = run_node[r];
        const int32_t c = run_pos[r + 1] - run_pos[r], gc = run_g[r + 1] - run_g[r];
        const int32_t eb = run_de[r], gb = run_dg[r];
        const bool big = c >= big_min;
        nrec[v] = make_int4(eb, eb + c, eb + (int32_t)region_cap(c, shift, big),
                            gb + (int32_t)region_cap(gc, shift, big) + 1);
        NodeRange x;
        x.g_lo = gb;
        x.g_hi = gb + gc;
        x.tb = 0;
        x.bs = 0;  // no time-bucket table (generation 0 is never a build's)
        x.t_first = E[run_pos[r]].ts;
        x.t_last = E[run_pos[r + 1] - 1].ts;
        ngr[v] = x;
        nbeg[v] = make_int2(eb, gb);
        ngo[gb + gc] = eb + c;
        act[r] = v;
    }
}

__global__ void k_nv_build_scatter(const Entry *__restrict__ E, const int32_t *__restrict__ run_of,
                                   const int32_t *__restrict__ fx, const int32_t *__restrict__ run_pos,
                                   const int32_t *__restrict__ run_g, const int32_t *__restrict__ run_de,
                                   const int32_t *__restrict__ run_dg, int64_t M, Entry *ent, int32_t *ngo,
                                   int64_t *ngts)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = run_of[p];
        const int32_t i = (int32_t)p - run_pos[r];
        const Entry x = E[p];
        const int32_t e = run_de[r] + i;
        ent[e] = x;
        if (fx[p + 1] != fx[p]) {
            const int32_t g = run_dg[r] + (fx[p] - run_g[r]);
            ngts[g] = x.ts;
            ngo[g] = e;
        }
    }
}

// ----------------------------------------------------------- batch append

// Per-node counts of the evicted entries (ev[v] += entries of v; each node
// that gets its first count is listed once in ev_nodes).  A Zipf stream puts
// most entries on a few hubs, and per-warp atomics on one hub's counter
// serialise at L2, so each block first sums its contiguous share of the
// items in a shared-memory table (warp peers combined by __match_any_sync,
// open addressing over EV_SLOTS keys, 16 probes) and adds each key's total
// once; a key that finds no slot goes straight to the global counter.
constexpr int EV_SLOTS = 2048;
constexpr int EV_PROBES = 16;

__device__ __forceinline__ void ev_add(int32_t v, int32_t cnt, int32_t *ev, int32_t *ev_nodes, NvCounters *c)
{
    const int32_t old = atomicAdd(&ev[v], cnt);
    if (old == 0) ev_nodes[atomicAdd(&c->n_ev_nodes, 1ull)] = v;
}

__global__ void __launch_bounds__(256) k_nv_evict_count(Items it, int64_t items, int64_t N, int32_t *ev,
                                                        int32_t *ev_nodes, NvCounters *c)
{
    __shared__ int32_t s_key[EV_SLOTS];
    __shared__ int32_t s_cnt[EV_SLOTS];
    for (int i = threadIdx.x; i < EV_SLOTS; i += blockDim.x) {
        s_key[i] = -1;
        s_cnt[i] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t per = (items + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per;
    const int64_t b1 = min(items, b0 + per);
    // the warp's hot key (the first key that filled 8 or more lanes) and its
    // running count, kept in registers (the same in every lane) and added to
    // the counter once at the end
    int32_t hot = -1, hot_cnt = 0;
    constexpr int U = 4;  // items per thread whose ids are loaded together
    // the next U items' ids are in flight while the current ones are counted
    auto load = [&](int64_t base, int32_t *vu) {
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t i = base + u * blockDim.x + threadIdx.x;
            vu[u] = i < b1 ? (int32_t)it.key(i) : 0;
        }
    };
    int32_t vn[U];
    load(b0, vn);
    for (int64_t base = b0; base < b1; base += (int64_t)U * blockDim.x) {
        int32_t vu[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            vu[u] = -1;
            if (base + u * blockDim.x + threadIdx.x < b1) {
                vu[u] = vn[u];
                if (vu[u] < 0 || vu[u] >= N) {
                    atomicOr(&c->status, 1ull << 0);
                    vu[u] = -1;
                }
            }
        }
        load(base + (int64_t)U * blockDim.x, vn);
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int32_t v = vu[u];
            const unsigned peers = __match_any_sync(0xffffffffu, v);
            if (hot < 0) {
                // claim the hot key: the lowest lane of a group of 8 or more
                const unsigned big = __ballot_sync(0xffffffffu, v >= 0 && __popc(peers) >= 8 && lane == __ffs(peers) - 1);
                if (big) hot = __shfl_sync(0xffffffffu, v, __ffs(big) - 1);
            }
            hot_cnt += __popc(__ballot_sync(0xffffffffu, v >= 0 && v == hot));  // the same in every lane
            if (v >= 0 && v == hot) continue;  // the next item of this thread
            if (v >= 0 && lane == __ffs(peers) - 1) {
                const int32_t cnt = __popc(peers);
                const uint32_t h0 = ((uint32_t)v * 2654435761u) >> 21;  // 11 bits: EV_SLOTS
                bool done = false;
                for (int p = 0; p < EV_PROBES && !done; p++) {
                    const int slot = (int)((h0 + (uint32_t)p) & (EV_SLOTS - 1));
                    int32_t k = s_key[slot];
                    if (k == -1) k = atomicCAS(&s_key[slot], -1, v);
                    if (k == -1 || k == v) {
                        atomicAdd(&s_cnt[slot], cnt);
                        done = true;
                    }
                }
                if (!done) ev_add(v, cnt, ev, ev_nodes, c);
            }
        }
    }
    if (lane == 0 && hot >= 0 && hot_cnt > 0) ev_add(hot, hot_cnt, ev, ev_nodes, c);
    __syncthreads();
    for (int i = threadIdx.x; i < EV_SLOTS; i += blockDim.x)
        if (s_key[i] >= 0) ev_add(s_key[i], s_cnt[i], ev, ev_nodes, c);
}

// Node v drops its entries before e_lo (r: its record) from the front of its
// region; returns the groups it lost.
__device__ __forceinline__ int32_t evict_node(int32_t v, int4 r, int32_t e_lo, int4 *nrec, NodeRange *ngr,
                                              int32_t *ngo, const int64_t *__restrict__ ngts, int32_t *nev)
{
    const int32_t gx = ngr[v].g_lo, gy = ngr[v].g_hi;
    int32_t ng;
    if (e_lo == r.y) {
        ng = gy;
    } else {
        // first group whose range ends after e_lo (ngo[gy] = r.y > e_lo):
        // the group starts grow about linearly with the group index (a hub's
        // groups hold about one entry each), so the first probes
        // interpolate, then the search bisects
        int32_t lo = gx, hi = gy - 1;
        int64_t vlo = ngo[lo], vhi = ngo[hi + 1];  // start of group lo, end of group hi
        for (int step = 0; lo < hi; step++) {
            int32_t mid = lo + ((hi - lo) >> 1);
            if (step < 4 && hi - lo > 16 && vhi > vlo) {
                const int64_t est = lo + (e_lo - vlo) * (int64_t)(hi + 1 - lo) / (vhi - vlo);
                mid = (int32_t)min(max(est, (int64_t)lo), (int64_t)(hi - 1));
            }
            const int32_t x = ngo[mid + 1];
            if (x > e_lo) {
                hi = mid;
                vhi = x;
            } else {
                lo = mid + 1;
                vlo = x;
            }
        }
        ng = lo;
        ngo[ng] = e_lo;  // the first kept group may have lost a prefix
        ngr[v].t_first = ngts[ng];
    }
    nev[v] += ng - gx;  // the node's group numbering origin moves with it (time-bucket table reuse)
    r.x = e_lo;
    nrec[v] = r;
    ngr[v].g_lo = ng;
    return ng - gx;
}

// Every node that lost entries drops them from the front of its region.
__global__ void k_nv_evict_apply(const int32_t *__restrict__ ev_nodes, int32_t *ev, int4 *nrec, NodeRange *ngr,
                                 int32_t *ngo, const int64_t *__restrict__ ngts, int32_t *nev, NvCounters *c)
{
    const int64_t n = (int64_t)c->n_ev_nodes;
    long long removed = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ev_nodes[j];
        const int32_t k = ev[v];
        ev[v] = 0;
        const int4 r = nrec[v];
        int32_t e_lo = r.x + k;
        if (k <= 0 || e_lo > r.y) {
            atomicOr(&c->status, 1ull << 1);
            e_lo = min(max(e_lo, r.x), r.y);
        }
        removed += evict_node(v, r, e_lo, nrec, ngr, ngo, ngts, nev);
    }
    removed = warp_sum((unsigned long long)removed);
    if ((threadIdx.x & 31) == 0 && removed) atomicAdd((unsigned long long *)&c->gn_delta, (unsigned long long)-removed);
}

// The same eviction without reading the evicted edges, for streams whose
// active nodes are far fewer than the evicted entries (a Zipf stream: tens
// of thousands of nodes against 10M entries per batch): within a node the
// entries ascend in store position, so each active node finds its first
// entry at or after the new store head (cut) by a search over its own
// entries, interpolating first (a hub's positions grow about linearly).
// The entries removed are summed and checked against the evicted count.
__global__ void k_nv_evict_scan(const int32_t *__restrict__ act, int64_t n_act, uint32_t cut,
                                const Entry *__restrict__ ent, int4 *nrec, NodeRange *ngr, int32_t *ngo,
                                const int64_t *__restrict__ ngts, int32_t *nev, NvCounters *c)
{
    long long removed_g = 0;
    unsigned long long removed_e = 0, nodes = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_act; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = act[j];
        const int4 r = nrec[v];
        if (r.x >= r.y) continue;
        auto rel = [&](int32_t e) { return (int32_t)((uint32_t)ent[e].slot - cut); };
        const int32_t r0 = rel(r.x);
        if (r0 >= 0) continue;  // its oldest entry is kept
        int32_t e_lo;
        const int32_t r1 = rel(r.y - 1);
        if (r1 < 0) {
            e_lo = r.y;  // every entry goes
        } else {
            // rel(lo) < 0 <= rel(hi)
            int32_t lo = r.x, hi = r.y - 1;
            int64_t vlo = r0, vhi = r1;
            for (int step = 0; hi - lo > 1; step++) {
                int32_t mid = lo + ((hi - lo) >> 1);
                if (step < 4 && hi - lo > 16 && vhi > vlo) {
                    const int64_t est = lo + (0 - vlo) * (int64_t)(hi - lo) / (vhi - vlo);
                    mid = (int32_t)min(max(est, (int64_t)lo + 1), (int64_t)(hi - 1));
                }
                const int32_t x = rel(mid);
                if (x < 0) {
                    lo = mid;
                    vlo = x;
                } else {
                    hi = mid;
                    vhi = x;
                }
            }
            e_lo = hi;
        }
        removed_e += (unsigned long long)(e_lo - r.x);
        nodes++;
        removed_g += evict_node(v, r, e_lo, nrec, ngr, ngo, ngts, nev);
    }
    removed_g = warp_sum((unsigned long long)removed_g);
    removed_e = warp_sum(removed_e);
    nodes = warp_sum(nodes);
    if ((threadIdx.x & 31) == 0) {
        if (removed_g) atomicAdd((unsigned long long *)&c->gn_delta, (unsigned long long)-removed_g);
        if (removed_e) atomicAdd(&c->ev_removed, removed_e);
        if (nodes) atomicAdd(&c->n_ev_nodes, nodes);
    }
}

// Batch-local node ids, so that the batch's node sort needs only as many
// key bits as the batch has distinct nodes.  The ids are exactly 0 ..
// distinct - 1: a warp's peers elect one leader per node, and a leader that
// finds the node unclaimed takes it with a compare-and-swap (0 -> -1) before
// it draws the next id (drawing first, as every racing warp of a hub would,
// spends ids that no node keeps, and a sparser id range costs sort passes).
// touched[id] names the node of each id; the sort's first histogram pass
// looks each entry's id up once every claim is done.
__global__ void k_nv_claim(Items it, int64_t nbe, int32_t *dense, int32_t *touched, NvCounters *c)
{
    const int lane = threadIdx.x & 31;
    constexpr int U = 4;  // entries per thread whose ids are loaded together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count (every lane takes part in the match)
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; base < nbe;
         base += stride * U) {
        int32_t v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t j = base + u * stride + lane;
            v[u] = j < nbe ? (int32_t)it.key(j) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned peers = __match_any_sync(0xffffffffu, v[u]);
            // a stale 0 from the cached read only costs a compare-and-swap that fails
            if (v[u] >= 0 && lane == __ffs(peers) - 1 && dense[v[u]] == 0 && atomicCAS(&dense[v[u]], 0, -1) == 0) {
                const int32_t id = (int32_t)atomicAdd(&c->n_dense, 1ull);
                touched[id] = v[u];
                dense[v[u]] = id + 1;
            }
        }
    }
}

__global__ void k_iota(uint32_t *v, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (uint32_t)i;
}

__global__ void k_nv_dense_reset(const int32_t *__restrict__ touched, const NvCounters *c, int32_t *dense)
{
    const int64_t n = (int64_t)c->n_dense;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = touched[i];
        if (v >= 0) dense[v] = 0;
    }
}

// The first sort pass's histogram reads each entry's batch-local id from the
// id table (dense[v] - 1; the batch's few thousand nodes keep their words in
// cache) and keeps it in ids[]; the first scatter pass reads ids[] (the
// table lookups had doubled that pass's time).
struct DenseLoader {
    Items it;
    const int32_t *dense;
    uint32_t *ids;
    __device__ __forceinline__ uint32_t key(int64_t i) const { return (uint32_t)(__ldg(dense + (int32_t)it.key(i)) - 1); }
    __device__ __forceinline__ void note(int64_t i, uint32_t k) const { ids[i] = k; }
};

struct NotedIdLoader {
    const uint32_t *ids;
    __device__ __forceinline__ uint32_t key(int64_t i) const { return ids[i]; }
    __device__ __forceinline__ uint32_t val(int64_t i) const { return (uint32_t)i; }
};

// Node runs and new groups of the batch's entries in (node, ts, arrival)
// order (kb: batch-local node ids; the run and group starts come as one byte
// per entry from k_nv_entries_runs, groups as of after the eviction: bit 0 a
// run start, bit 1 a group start).  A byte scan (each thread reads 16 flags
// with one load) that writes the run records and each tile's prefix; the
// scatter and the weight update derive every entry's run and group from the
// same bytes (RunTile), so no per-entry array is written.  Gathering each
// timestamp through the sort's index had cost four scattered loads per
// entry, and the generic scan over one byte per element 44 instructions per
// element.
struct AppendRunBytes {
    const uint8_t *flags;  // 16-byte aligned
    int64_t n;
    const uint32_t *kb;
    const int32_t *touched;
    int32_t *run_node, *run_pos, *run_g;
    uint64_t *tile_prefix;  // per tile: runs (high) and groups (low) before it
    struct Stage {};
    __host__ __device__ int64_t tiles() const { return n > 0 ? (n + BSCAN_TILE - 1) / BSCAN_TILE : 0; }
    __device__ __forceinline__ uint4 load(int64_t u0) const
    {
        return u0 < n ? __ldg(reinterpret_cast<const uint4 *>(flags + u0)) : make_uint4(0, 0, 0, 0);
    }
    __device__ __forceinline__ uint64_t sum16(uint4 w, int64_t u0) const
    {
        const uint32_t v = valid16(u0, 0, n);
        return ((uint64_t)__popc(byte_bits16(w, 0) & v) << 32) | (uint64_t)__popc(byte_bits16(w, 1) & v);
    }
    __device__ __forceinline__ void emit16(uint4 w, int64_t u0, uint64_t ex, uint64_t tile_ex, uint64_t,
                                           Stage &) const
    {
        if (threadIdx.x == 0) tile_prefix[u0 / BSCAN_TILE] = tile_ex;
        const uint32_t v = valid16(u0, 0, n);
        uint32_t rm = byte_bits16(w, 0) & v;
        if (!rm) return;
        const uint32_t gm = byte_bits16(w, 1) & v;
        uint32_t R = (uint32_t)(ex >> 32);
        const uint32_t G = (uint32_t)ex;
        while (rm) {  // a node run starts at each set bit
            const int k = __ffs(rm) - 1;
            rm &= rm - 1;
            const int64_t p = u0 + k;
            run_node[R] = touched[kb[p]];
            run_pos[R] = (int32_t)p;
            run_g[R] = (int32_t)(G + (uint32_t)__popc(gm & ((1u << k) - 1u)));
            R++;
        }
    }
};

// One thread per node run: room in place; else, when the evicted front of
// the node's own regions can take its live items without overlapping them, a
// move back to the regions' start (a sliding window's steady state: no pool
// space is used); else fresh regions from the pools and a move.
// Big nodes (a Zipf hub) slide their live range back to the front of their
// regions every few dozen batches (a sliding window's steady state), a copy
// of all their entries and groups in one batch.  Instead, in the batches
// before the one that no longer fits, each copies a share of the range that
// will then be live (from its predicted start) to the front, and the batch
// that no longer fits copies the rest and moves the node onto the copy.
constexpr int NV_MIRRORS = 64;               // big nodes copying ahead at once
constexpr int64_t NV_MIRROR_BATCHES = 16;    // batches ahead of the slide

// The slot of node v, or -1.  All NV_MIRRORS loads issue together (an early
// exit made them a chain of dependent L2 loads on the hub's thread, the
// reserve kernel's critical path); only v's own thread writes v's slot.
__device__ __forceinline__ int mirror_find(const NvMirror *mir, int32_t v)
{
    int found = -1;
#pragma unroll
    for (int i = 0; i < NV_MIRRORS; i++)
        if (__ldcg(&mir[i].node) == v) found = i;
    return found;
}

__global__ void k_nv_reserve(const int32_t *__restrict__ run_node, const int32_t *__restrict__ run_pos,
                             const int32_t *__restrict__ run_g, const uint64_t *__restrict__ tot, int shift,
                             int64_t e_cap, int64_t g_cap, int4 *nrec, NodeRange *ngr, int2 *nbeg, int32_t *ngo,
                             int32_t *act, int64_t act_cap, Reloc *reloc, int32_t *run_de, int32_t *run_dg,
                             NvMirror *mir, int32_t mirror_min, NvCounters *c)
{
    const int64_t R = (int64_t)(*tot >> 32);
    long long added = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = run_node[r];
        const int32_t cnt = run_pos[r + 1] - run_pos[r], gc = run_g[r + 1] - run_g[r];
        int4 rec = nrec[v];
        int2 g = make_int2(ngr[v].g_lo, ngr[v].g_hi);
        const bool fresh = rec.z == 0;
        if (fresh) {
            const unsigned long long a = atomicAdd(&c->n_act, 1ull);
            if ((int64_t)a < act_cap) act[a] = v;
            else atomicOr(&c->status, 1ull << 2);
        }
        const int32_t live_e = rec.y - rec.x, live_g = g.y - g.x;
        int32_t d_e, d_g;
        if (!fresh && (int64_t)rec.y + cnt <= rec.z && (int64_t)g.y + gc + 1 <= rec.w) {
            d_e = rec.y;
            d_g = g.y;
            if (live_e >= mirror_min) {
                // batches like this one that fit, this one included
                const int64_t fits = min((int64_t)(rec.z - rec.y) / max(cnt, 1),
                                         (int64_t)(rec.w - g.y - 1) / max(gc, 1));
                const int2 beg = nbeg[v];
                int m = mirror_find(mir, v);
                if (m < 0 && fits <= NV_MIRROR_BATCHES) {
                    // the range live at the slide starts about fits - 1
                    // batches of groups on (this batch's groups as the rate)
                    const int32_t gm = (int32_t)min((int64_t)g.y, (int64_t)g.x + (fits - 1) * (int64_t)gc);
                    const int32_t xm = gm < g.y ? ngo[gm] : rec.y;
                    for (int i = (int)((uint32_t)v % NV_MIRRORS), k = 0; k < NV_MIRRORS && m < 0;
                         k++, i = (i + 1) % NV_MIRRORS)
                        if (atomicCAS(&mir[i].node, -1, v) == -1) {
                            mir[i].x_m = xm;
                            mir[i].g_m = gm;
                            mir[i].c_e = 0;
                            mir[i].c_g = 0;
                            m = i;
                        }
                }
                if (m >= 0) {
                    // this batch's share, written below the live range only
                    NvMirror q = mir[m];
                    const int64_t fe = max(fits, (int64_t)1);
                    int64_t se = ((int64_t)rec.y - (q.x_m + q.c_e) + fe - 1) / fe;
                    int64_t sg = ((int64_t)g.y - (q.g_m + q.c_g) + fe - 1) / fe;
                    se = max((int64_t)0, min(se, (int64_t)rec.x - (beg.x + q.c_e)));
                    sg = max((int64_t)0, min(sg, (int64_t)g.x - (beg.y + q.c_g)));
                    if (se > 0 || sg > 0) {
                        atomicAdd(&c->moved_e, (unsigned long long)se);
                        atomicAdd(&c->moved_g, (unsigned long long)sg);
                        const unsigned long long t = atomicAdd(&c->n_reloc, 1ull);
                        reloc[t] = Reloc{q.x_m + q.c_e, (int32_t)se, beg.x + q.c_e, q.g_m + q.c_g, (int32_t)sg,
                                         beg.y + q.c_g};
                        mir[m].c_e = q.c_e + (int32_t)se;
                        mir[m].c_g = q.c_g + (int32_t)sg;
                    }
                }
            }
            rec.y += cnt;
        } else {
            const int2 beg = fresh ? make_int2(0, 0) : nbeg[v];
            bool switched = false;
            // the regions change here: a copy made ahead (whatever the node's
            // size now) is used or dropped
            const int ms = fresh ? -1 : mirror_find(mir, v);
            if (ms >= 0) {
                // the copy made ahead holds [x_m, x_m + c_e) and [g_m, g_m + c_g)
                const NvMirror q = mir[ms];
                const int64_t ne = (int64_t)rec.y - q.x_m, ng = (int64_t)g.y - q.g_m;
                if (q.x_m <= rec.x && q.g_m <= g.x && beg.x + ne <= (int64_t)q.x_m + q.c_e &&
                    beg.y + ng <= (int64_t)q.g_m + q.c_g && ne + cnt <= (int64_t)rec.z - beg.x &&
                    ng + gc + 1 <= (int64_t)rec.w - beg.y) {
                    const int32_t re = (int32_t)(ne - q.c_e), rg = (int32_t)(ng - q.c_g);
                    if (re > 0 || rg > 0) {
                        atomicAdd(&c->moved_e, (unsigned long long)max(re, 0));
                        atomicAdd(&c->moved_g, (unsigned long long)max(rg, 0));
                        const unsigned long long t = atomicAdd(&c->n_reloc, 1ull);
                        reloc[t] = Reloc{q.x_m + q.c_e, max(re, 0), beg.x + q.c_e, q.g_m + q.c_g, max(rg, 0),
                                         beg.y + q.c_g};
                    }
                    const int32_t nx = beg.x + (rec.x - q.x_m), gx = beg.y + (g.x - q.g_m);
                    // the first live group may have lost a prefix since it was copied
                    ngo[gx] = nx;
                    d_e = beg.x + (int32_t)ne;
                    d_g = beg.y + (int32_t)ng;
                    rec = make_int4(nx, d_e + cnt, rec.z, rec.w);
                    g.x = gx;
                    switched = true;
                    atomicAdd(&c->mir_switched, 1ull);
                }
                mir[ms].node = -1;
            }
            if (!switched) {
                const bool slide = !fresh && rec.x - beg.x >= live_e && g.x - beg.y >= live_g &&
                                   (int64_t)live_e + cnt <= rec.z - beg.x && (int64_t)live_g + gc + 1 <= rec.w - beg.y;
                int64_t ecap, gcap;
                unsigned long long eb, gb;
                if (slide) {
                    eb = (unsigned long long)beg.x;
                    gb = (unsigned long long)beg.y;
                    ecap = rec.z - beg.x;
                    gcap = rec.w - beg.y;
                } else {
                    const bool big = (int64_t)live_e + cnt >= mirror_min;
                    ecap = region_cap((int64_t)live_e + cnt, shift, big);
                    gcap = region_cap((int64_t)live_g + gc, shift, big) + 1;
                    eb = atomicAdd(&c->e_top, (unsigned long long)ecap);
                    gb = atomicAdd(&c->g_top, (unsigned long long)gcap);
                    if ((int64_t)eb + ecap > e_cap || (int64_t)gb + gcap > g_cap) {
                        atomicOr(&c->overflow, 1ull);
                        run_de[r] = -1;
                        continue;
                    }
                    nbeg[v] = make_int2((int32_t)eb, (int32_t)gb);
                }
                if (live_e > 0 || live_g > 0) {
                    atomicAdd(&c->moved_e, (unsigned long long)live_e);
                    atomicAdd(&c->moved_g, (unsigned long long)live_g);
                    const unsigned long long t = atomicAdd(&c->n_reloc, 1ull);
                    reloc[t] = Reloc{rec.x, live_e, (int32_t)eb, g.x, live_g, (int32_t)gb};
                }
                d_e = (int32_t)eb + live_e;
                d_g = (int32_t)gb + live_g;
                rec = make_int4((int32_t)eb, d_e + cnt, (int32_t)(eb + ecap), (int32_t)(gb + gcap));
                g.x = (int32_t)gb;
            }
        }
        g.y = d_g + gc;
        nrec[v] = rec;
        ngr[v].g_lo = g.x;
        ngr[v].g_hi = g.y;
        // the slot after the last group (= rec.y) is written with the batch's
        // groups, after any move has read the old groups
        run_de[r] = d_e;
        run_dg[r] = d_g;
        added += gc;
    }
    added = warp_sum((unsigned long long)added);
    if ((threadIdx.x & 31) == 0 && added) {
        atomicAdd((unsigned long long *)&c->gn_delta, (unsigned long long)added);
        atomicAdd(&c->g_added, (unsigned long long)added);
    }
}

// Chunks of each move, over a bound on the moves (the count is read on the
// device, so the host needs no round trip between the reservation and the
// moves).
struct RelocChunkOp {
    const Reloc *reloc;
    int32_t *cbase;
    const NvCounters *c;
    __device__ __forceinline__ uint64_t value(int64_t t) const
    {
        if (t >= (int64_t)c->n_reloc || c->overflow) return 0;
        const Reloc x = reloc[t];
        return (uint64_t)((max(x.n_e, x.n_g) + RELOC_CHUNK - 1) / RELOC_CHUNK);
    }
    __device__ __forceinline__ void emit(int64_t t, uint64_t, uint64_t ex) const { cbase[t] = (int32_t)ex; }
};

// One warp per chunk of a move: entries copied, group timestamps copied,
// group starts rebased to the new entry region.
__global__ void k_nv_reloc(const Reloc *__restrict__ reloc, const int32_t *__restrict__ cbase, const NvCounters *c,
                           const uint64_t *__restrict__ tot, Entry *ent, int32_t *ngo, int64_t *ngts, double *gw)
{
    if (c->overflow) return;  // the batch rebuilds the view instead
    const int lane = threadIdx.x & 31;
    const int64_t n_reloc = (int64_t)c->n_reloc;
    const int64_t nch = (int64_t)*tot;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < nch; ch += warps) {
        int64_t lo = 0, hi = n_reloc - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (cbase[mid] <= ch) lo = mid;
            else hi = mid - 1;
        }
        const Reloc x = reloc[lo];
        const int32_t off = (int32_t)(ch - cbase[lo]) * RELOC_CHUNK;
        const int32_t e_end = min(x.n_e, off + RELOC_CHUNK);
        for (int32_t i = off + lane; i < e_end; i += 32) ent[x.new_e + i] = ent[x.old_e + i];
        const int32_t g_end = min(x.n_g, off + RELOC_CHUNK);
        for (int32_t i = off + lane; i < g_end; i += 32) {
            ngts[x.new_g + i] = ngts[x.old_g + i];
            ngo[x.new_g + i] = ngo[x.old_g + i] - x.old_e + x.new_e;
            if (gw) gw[x.new_g + i] = gw[x.old_g + i];  // group weights move with their groups
        }
    }
}

// Four blocks per tile of BSCAN_TILE entries, each writing a quarter (four
// entries per thread, loaded before the tile's flags are scanned): each
// entry's run and group come from the flag bytes (RunTile).  Short blocks
// keep the last wave small (one block per tile left a fifth wave of a few
// blocks at 10M entries).
constexpr int SCATTER_SPLIT = 4;

__global__ void __launch_bounds__(BSCAN_THREADS)
    k_nv_scatter(const Entry *__restrict__ E, const uint8_t *__restrict__ flags, int64_t nbe,
                 const uint64_t *__restrict__ tile_prefix, const int32_t *__restrict__ run_pos,
                 const int32_t *__restrict__ run_g, const int32_t *__restrict__ run_de,
                 const int32_t *__restrict__ run_dg, const int32_t *__restrict__ run_node, int64_t e_cap,
                 int64_t g_cap, Entry *ent, int32_t *ngo, int64_t *ngts, NodeRange *ngr, NvCounters *c)
{
    if (c->overflow) return;  // a pool could not serve a region: the batch rebuilds the view instead
    constexpr int U = 16 / SCATTER_SPLIT;
    __shared__ RunTile sm;
    const int64_t t = blockIdx.x / SCATTER_SPLIT, p0 = t * BSCAN_TILE;
    const int k0 = (int)(blockIdx.x % SCATTER_SPLIT) * U;
    Entry xs[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int64_t p = p0 + (k0 + u) * BSCAN_THREADS + threadIdx.x;
        if (p < nbe) xs[u] = E[p];
    }
    run_tile_load(sm, flags, nbe, t, tile_prefix[t]);
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int j = (k0 + u) * BSCAN_THREADS + threadIdx.x;
        const int64_t p = p0 + j;
        if (p >= nbe) break;
        const RunAt a = run_tile_at(sm, j);
        const int32_t r = a.r;
        const int32_t de = run_de[r];
        const int32_t i = (int32_t)p - run_pos[r];
        const int64_t e = (int64_t)de + i;
        if (de < 0 || e >= e_cap) {
            atomicOr(&c->status, 1ull << 3);
            continue;
        }
        const Entry x = xs[u];
        ent[e] = x;
        // the node record's first / last group timestamps
        const bool last = p + 1 == run_pos[r + 1];
        if (a.rs) {
            const int32_t v = run_node[r];
            if (ngr[v].g_lo == run_dg[r]) ngr[v].t_first = x.ts;  // no live group before the batch
        }
        if (last) ngr[run_node[r]].t_last = x.ts;
        if (a.gs) {
            const int64_t g = (int64_t)run_dg[r] + (a.g - run_g[r]);
            if (g < 0 || g >= g_cap) {
                atomicOr(&c->status, 1ull << 4);
                continue;
            }
            ngts[g] = x.ts;
            ngo[g] = (int32_t)e;
        }
        if (last) {  // the node's new end after its last group
            const int64_t gs = (int64_t)run_dg[r] + (run_g[r + 1] - run_g[r]);
            if (gs < 0 || gs >= g_cap) {
                atomicOr(&c->status, 1ull << 5);
                continue;
            }
            ngo[gs] = (int32_t)(e + 1);
        }
    }
}

// ------------------------------------------------------------------ exports

struct CountOp {
    const int4 *nrec;
    const NodeRange *ngr;
    int64_t N;
    int groups;
    int32_t *out;
    __device__ __forceinline__ uint64_t value(int64_t v) const
    {
        if (v >= N) return 0;
        return groups ? (uint64_t)(ngr[v].g_hi - ngr[v].g_lo) : (uint64_t)(nrec[v].y - nrec[v].x);
    }
    __device__ __forceinline__ void emit(int64_t v, uint64_t, uint64_t ex) const { out[v] = (int32_t)ex; }
};

// One warp per node: its entries' store positions (node order) or its group
// starts (canonical offsets), at the node's canonical place.
__global__ void k_nv_export(const int4 *__restrict__ nrec, const NodeRange *__restrict__ ngr,
                            const int32_t *__restrict__ off, const int32_t *__restrict__ gidx,
                            const Entry *__restrict__ ent, const int32_t *__restrict__ ngo, int64_t N,
                            uint32_t slot_base, int groups, int32_t *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < N; v += warps) {
        const int4 r = nrec[v];
        if (!groups) {
            for (int32_t i = lane; i < r.y - r.x; i += 32)
                out[off[v] + i] = (int32_t)((uint32_t)ent[r.x + i].slot - slot_base);
        } else {
            const int32_t gx = ngr[v].g_lo, gy = ngr[v].g_hi;
            for (int32_t i = lane; i < gy - gx; i += 32) out[gidx[v] + i] = off[v] + (ngo[gx + i] - r.x);
        }
    }
}

unsigned grid_for(tempest_t *h, int64_t n, int threads = 256)
{
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)h->num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b < 1 ? 1 : b;
}

uint32_t slot_base(const tempest_t *h, int64_t idx)
{
    const uint64_t p = (uint64_t)(h->s_base + idx);
    return (uint32_t)(h->directed ? p : 2 * p);
}

Items items_at(const tempest_t *h, int buf, int64_t idx)
{
    return Items{h->st_src[buf].as<int32_t>() + idx, h->st_dst[buf].as<int32_t>() + idx,
                 h->st_ts[buf].as<int64_t>() + idx, h->directed};
}

int ensure_runs(tempest_t *h, int64_t items, int64_t runs)
{
    int rc;
    const size_t iz = (size_t)(items + 1), rz = (size_t)(runs + 1);
    if ((rc = ensure(h, h->run_of, sizeof(int32_t) * iz, true))) return rc;
    if ((rc = ensure(h, h->fx, sizeof(int32_t) * iz, true))) return rc;
    if ((rc = ensure(h, h->run_node, sizeof(int32_t) * rz, true))) return rc;
    if ((rc = ensure(h, h->run_pos, sizeof(int32_t) * rz, true))) return rc;
    if ((rc = ensure(h, h->run_g, sizeof(int32_t) * rz, true))) return rc;
    if ((rc = ensure(h, h->run_de, sizeof(int32_t) * rz, true))) return rc;
    if ((rc = ensure(h, h->run_dg, sizeof(int32_t) * rz, true))) return rc;
    for (int b = 0; b < 2; b++) {
        if ((rc = ensure(h, h->sk32[b], sizeof(uint32_t) * iz, true))) return rc;
        if ((rc = ensure(h, h->sv[b], sizeof(uint32_t) * iz, true))) return rc;
    }
    return TEMPEST_OK;
}

// Grows an array that must keep its contents (zero-filled tail).
int grow_keep(tempest_t *h, DBuf &b, size_t used, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return TEMPEST_OK;
    DBuf nb;
    std::swap(nb, b);  // b empty: ensure allocates fresh
    int rc = ensure(h, b, bytes + bytes / 4);
    if (rc) {
        std::swap(nb, b);
        return rc;
    }
    if (used && nb.p) cudaMemcpyAsync(b.p, nb.p, used, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemsetAsync(static_cast<char *>(b.p) + used, 0, b.bytes - used, h->stream);
    release(h, nb);
    return TEMPEST_OK;
}

}  // namespace

// Per-node arrays cover node slots [0, N]: existing records kept, new ones
// empty, the per-node eviction counters zero.
int nv_ensure_nodes(tempest_t *h, int64_t N)
{
    const int64_t need = N + 1;
    if (need <= h->nrec_n && h->ngr.p && h->nrec.p && h->ev.p && h->act.p && h->dense.p && h->nbeg.p && h->nev.p)
        return TEMPEST_OK;
    int rc;
    const size_t used = (size_t)h->nrec_n;
    if ((rc = grow_keep(h, h->nrec, sizeof(int4) * used, sizeof(int4) * (size_t)need))) return rc;
    if ((rc = grow_keep(h, h->ngr, sizeof(NodeRange) * used, sizeof(NodeRange) * (size_t)need))) return rc;
    if ((rc = grow_keep(h, h->ev, sizeof(int32_t) * used, sizeof(int32_t) * (size_t)need))) return rc;
    if ((rc = grow_keep(h, h->act, sizeof(int32_t) * (size_t)h->n_act, sizeof(int32_t) * (size_t)need))) return rc;
    if ((rc = grow_keep(h, h->dense, sizeof(int32_t) * used, sizeof(int32_t) * (size_t)need))) return rc;
    if ((rc = grow_keep(h, h->nbeg, sizeof(int2) * used, sizeof(int2) * (size_t)need))) return rc;
    if ((rc = grow_keep(h, h->nev, sizeof(int32_t) * used, sizeof(int32_t) * (size_t)need))) return rc;
    int64_t cover = (int64_t)(h->nrec.bytes / sizeof(int4));
    cover = std::min(cover, (int64_t)(h->nbeg.bytes / sizeof(int2)));
    cover = std::min(cover, (int64_t)(h->dense.bytes / sizeof(int32_t)));
    cover = std::min(cover, (int64_t)(h->ngr.bytes / sizeof(NodeRange)));
    cover = std::min(cover, (int64_t)(h->ev.bytes / sizeof(int32_t)));
    cover = std::min(cover, (int64_t)(h->act.bytes / sizeof(int32_t)));
    cover = std::min(cover, (int64_t)(h->nev.bytes / sizeof(int32_t)));
    h->nrec_n = cover;
    return TEMPEST_OK;
}

// Whole view from the live store.
int nv_build(tempest_t *h)
{
    NvtxRange range("node view: rebuild");
    cudaStream_t st = h->stream;
    const int64_t m = h->s_hi - h->s_lo;
    const int64_t M = h->directed ? m : 2 * m;
    const int64_t N = h->N;
    int rc;
    if ((rc = nv_ensure_nodes(h, N))) return rc;
    if ((rc = ensure(h, h->nvc, sizeof(NvCounters)))) return rc;
    if ((rc = ensure(h, h->nv_mir, sizeof(NvMirror) * NV_MIRRORS))) return rc;
    cudaMemsetAsync(h->nv_mir.p, 0xff, sizeof(NvMirror) * NV_MIRRORS, st);  // no copies made ahead
    cudaMemsetAsync(h->nrec.p, 0, h->nrec.bytes, st);
    cudaMemsetAsync(h->ngr.p, 0, h->ngr.bytes, st);
    h->bkt_prev_ok = false;  // groups are renumbered: no table of an earlier build can be reused
    cudaMemsetAsync(h->nvc.p, 0, sizeof(NvCounters), st);
    h->n_act = 0;
    h->Gn = 0;
    h->M = M;
    h->pending_launches += 4;
    if (M == 0) {
        h->nv_ready = true;
        return cuda_check(h, cudaGetLastError(), "node view");
    }
    const int64_t runs_max = std::min(M, N);
    if ((rc = ensure_runs(h, M, runs_max))) return rc;
    if ((rc = ensure(h, h->nv_tmp, sizeof(Entry) * (size_t)M, true))) return rc;
    const Items it = items_at(h, h->cur, h->s_lo);
    uint32_t *kb[2] = {h->sk32[0].as<uint32_t>(), h->sk32[1].as<uint32_t>()};
    uint32_t *vb[2] = {h->sv[0].as<uint32_t>(), h->sv[1].as<uint32_t>()};
    int launches = 0;
    const int r = radix_sort_launch<uint32_t>(it, M, bits_for((uint64_t)(N > 0 ? N - 1 : 0)), kb, vb,
                                              h->hist.as<uint32_t>(), st, &launches);
    Entry *E = h->nv_tmp.as<Entry>();
    k_nv_entries<<<grid_for(h, M), 256, 0, st>>>(vb[r], it, M, slot_base(h, h->s_lo), E);
    uint64_t *part = h->partials.as<uint64_t>();
    BuildRunOp op{kb[r], E, h->run_of.as<int32_t>(), h->fx.as<int32_t>(), h->run_node.as<int32_t>(),
                  h->run_pos.as<int32_t>(), h->run_g.as<int32_t>()};
    int nb = scan_launch(op, M, part, st);
    k_nv_tail<<<1, 1, 0, st>>>(h->run_pos.as<int32_t>(), h->run_g.as<int32_t>(), h->fx.as<int32_t>(), part + nb, M);
    uint64_t *hp = static_cast<uint64_t *>(h->hstat);
    cudaMemcpyAsync(hp, part + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    h->pending_launches += launches + 5;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "node view runs"))) return rc;
    const int64_t S = (int64_t)(hp[0] >> 32), Gn = (int64_t)(uint32_t)hp[0];
    // region slack: halve it until the pools fit the int32 index range
    int shift = 0;
    while (shift < 4 && (M + (M >> shift) + (M >> (shift + 1)) + 16 * S + 1 >= (int64_t)INT32_MAX / 2 ||
                         Gn + (Gn >> shift) + (Gn >> (shift + 1)) + 17 * S + 1 >= (int64_t)INT32_MAX / 2))
        shift++;
    h->nv_shift = shift;
    CapOp cop{h->run_pos.as<int32_t>(), h->run_g.as<int32_t>(), shift, h->mirror_min, h->run_de.as<int32_t>(),
              h->run_dg.as<int32_t>()};
    nb = scan_launch(cop, S, part, st);
    cudaMemcpyAsync(hp, part + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "node view regions"))) return rc;
    const int64_t e_need = (int64_t)(uint32_t)hp[0], g_need = (int64_t)(hp[0] >> 32);
    // pools: the regions plus as much again for regions that move
    const int64_t e_cap = std::min((int64_t)INT32_MAX - 1, 2 * e_need + 4096);
    const int64_t g_cap = std::min((int64_t)INT32_MAX - 1, 2 * g_need + 4096);
    if (e_need >= e_cap || g_need >= g_cap)
        return fail(h, TEMPEST_ENOMEM, "node view: %lld entries exceed the int32 index range", (long long)M);
    if ((rc = ensure(h, h->ent, sizeof(Entry) * (size_t)e_cap))) return rc;
    if ((rc = ensure(h, h->ngo, sizeof(int32_t) * (size_t)g_cap))) return rc;
    if ((rc = ensure(h, h->ngts, sizeof(int64_t) * (size_t)g_cap))) return rc;
    h->e_cap = (int64_t)(h->ent.bytes / sizeof(Entry));
    h->g_cap = std::min((int64_t)(h->ngo.bytes / sizeof(int32_t)), (int64_t)(h->ngts.bytes / sizeof(int64_t)));
    h->e_cap = std::min(h->e_cap, (int64_t)INT32_MAX - 1);
    h->g_cap = std::min(h->g_cap, (int64_t)INT32_MAX - 1);
    k_nv_build_nodes<<<grid_for(h, S), 256, 0, st>>>(h->run_node.as<int32_t>(), h->run_pos.as<int32_t>(),
                                                     h->run_g.as<int32_t>(), h->run_de.as<int32_t>(),
                                                     h->run_dg.as<int32_t>(), E, S, shift, h->mirror_min,
                                                     h->nrec.as<int4>(),
                                                     h->ngr.as<NodeRange>(), h->nbeg.as<int2>(), h->ngo.as<int32_t>(),
                                                     h->act.as<int32_t>());
    k_nv_build_scatter<<<grid_for(h, M), 256, 0, st>>>(E, h->run_of.as<int32_t>(), h->fx.as<int32_t>(),
                                                       h->run_pos.as<int32_t>(), h->run_g.as<int32_t>(),
                                                       h->run_de.as<int32_t>(), h->run_dg.as<int32_t>(), M,
                                                       h->ent.as<Entry>(), h->ngo.as<int32_t>(),
                                                       h->ngts.as<int64_t>());
    NvCounters c0{};
    c0.e_top = (unsigned long long)e_need;
    c0.g_top = (unsigned long long)g_need;
    c0.n_act = (unsigned long long)S;
    cudaMemcpyAsync(h->nvc.p, &c0, sizeof(NvCounters), cudaMemcpyHostToDevice, st);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "node view build"))) return rc;
    h->pending_launches += 7;
    h->n_act = S;
    h->S = S;
    h->Gn = Gn;
    h->nv_ready = true;
    h->w_valid = false;  // new regions: the weights are recomputed for the next walks
    h->nv_rep.rebuilt = true;
    h->nv_rep.rb_entries = M;
    h->nv_rep.rb_passes = (bits_for((uint64_t)(N > 0 ? N - 1 : 0)) + RADIX_BITS - 1) / RADIX_BITS;
    h->nv_rep.rb_nodes = S;
    h->nv_rep.rb_groups = Gn;
    return TEMPEST_OK;
}

// Every buffer nv_append will need for a batch of nbk kept edges after
// evicting n_ev edges, allocated now (nv_append's own ensure calls then find
// them in place), so that an ingest whose memory runs short fails before it
// changes anything.  A pool that later proves too small still rebuilds.
int nv_prepare_append(tempest_t *h, int64_t n_ev, int64_t nbk, int64_t N_old, int64_t N_new)
{
    const int64_t ne = h->directed ? n_ev : 2 * n_ev, nbe = h->directed ? nbk : 2 * nbk;
    int rc;
    if ((rc = nv_ensure_nodes(h, N_new))) return rc;
    if ((rc = ensure(h, h->nvc, sizeof(NvCounters)))) return rc;
    if (ne > 0 && (rc = ensure(h, h->ev_nodes, sizeof(int32_t) * (size_t)std::min(ne, N_old + 1), true))) return rc;
    if (nbe > 0) {
        const int64_t runs_max = std::min(nbe, N_new);
        if ((rc = ensure_runs(h, nbe, runs_max))) return rc;
        if ((rc = ensure(h, h->reloc, sizeof(Reloc) * (size_t)(runs_max + 1), true))) return rc;
        if ((rc = ensure(h, h->nv_tmp, sizeof(int32_t) * (size_t)(runs_max + 1), true))) return rc;
        if ((rc = ensure(h, h->touched, sizeof(int32_t) * (size_t)nbe, true))) return rc;
        if ((rc = ensure(h, h->ent_tmp, sizeof(Entry) * (size_t)nbe, true))) return rc;
        if ((rc = ensure(h, h->nv_flags, (size_t)nbe, true))) return rc;
        if ((rc = ensure(h, h->nv_tex, sizeof(uint64_t) * (size_t)((nbe + BSCAN_TILE - 1) / BSCAN_TILE), true)))
            return rc;
    }
    return TEMPEST_OK;
}

// Queues the append of the store items of the edges [new_lo, new_lo + nbk)
// of the current buffer after evicting the n_ev oldest edges, whose
// endpoints are ev_src / ev_dst.  The node view's counters are read by the
// caller's next round trip and passed to nv_append_finish, which reports a
// pool that ran out (the caller then rebuilds the whole view).
int nv_append(tempest_t *h, const int32_t *ev_src, const int32_t *ev_dst, int64_t n_ev, int64_t new_lo, int64_t nbk,
              int64_t N_old)
{
    cudaStream_t st = h->stream;
    const int directed = h->directed;
    const int64_t N = h->N;
    const int64_t ne = directed ? n_ev : 2 * n_ev, nbe = directed ? nbk : 2 * nbk;
    int rc;
    NvtxStages stage;
    stage.next("node view: eviction");
    NvBatchReport &rep = h->nv_rep;
    rep.ev_entries = ne;
    rep.entries = nbe;
    if ((rc = nv_ensure_nodes(h, N))) return rc;
    if ((rc = ensure(h, h->nvc, sizeof(NvCounters)))) return rc;
    NvCounters *dc = h->nvc.as<NvCounters>();
    // keep the pool pointers and region count, reset the per-batch counters
    cudaMemsetAsync(&dc->gn_delta, 0, sizeof(NvCounters) - offsetof(NvCounters, gn_delta), st);
    cudaMemcpyAsync(&dc->n_act, &h->n_act, sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (ne > 0) {
        if ((rc = ensure(h, h->ev_nodes, sizeof(int32_t) * (size_t)std::min(ne, N_old + 1), true))) return rc;
        const Items ei{ev_src, ev_dst, nullptr, directed};
        for (cudaEvent_t &e : h->eev)
            if (!e) cudaEventCreate(&e);
        cudaEventRecord(h->eev[0], st);
        const bool scan = h->n_act > 0 && (h->evict_mode == 2 || (h->evict_mode == 0 && 8 * h->n_act < ne));
        if (scan) {
            // far fewer active nodes than evicted entries: each searches its
            // own entries for the new store head instead
            rep.ev_scanned = h->n_act;
            k_nv_evict_scan<<<grid_for(h, h->n_act), 256, 0, st>>>(
                h->act.as<int32_t>(), h->n_act, slot_base(h, h->s_lo), h->ent.as<Entry>(), h->nrec.as<int4>(),
                h->ngr.as<NodeRange>(), h->ngo.as<int32_t>(), h->ngts.as<int64_t>(), h->nev.as<int32_t>(), dc);
            h->pending_launches += 1;
        } else {
            // contiguous shares of at least 2048 items per block, at most 8 blocks per SM
            const int64_t eg = std::max<int64_t>(1, std::min<int64_t>((ne + 2047) / 2048, 8 * (int64_t)h->num_sms));
            k_nv_evict_count<<<(unsigned)eg, 256, 0, st>>>(ei, ne, N_old, h->ev.as<int32_t>(),
                                                           h->ev_nodes.as<int32_t>(), dc);
            k_nv_evict_apply<<<grid_for(h, std::min(ne, N_old)), 256, 0, st>>>(
                h->ev_nodes.as<int32_t>(), h->ev.as<int32_t>(), h->nrec.as<int4>(), h->ngr.as<NodeRange>(),
                h->ngo.as<int32_t>(), h->ngts.as<int64_t>(), h->nev.as<int32_t>(), dc);
            h->pending_launches += 2;
        }
        cudaEventRecord(h->eev[1], st);
        h->eev_valid = true;
    }
    if (nbe > 0) {
        const int64_t runs_max = std::min(nbe, N);
        if ((rc = ensure_runs(h, nbe, runs_max))) return rc;
        if ((rc = ensure(h, h->reloc, sizeof(Reloc) * (size_t)(runs_max + 1), true))) return rc;
        if ((rc = ensure(h, h->nv_tmp, sizeof(int32_t) * (size_t)(runs_max + 1), true))) return rc;
        const Items it = items_at(h, h->cur, new_lo);
        // batch-local node ids (the first sort pass reads them from dense[])
        stage.next("node view: batch ids and sort");
        if ((rc = ensure(h, h->touched, sizeof(int32_t) * (size_t)nbe, true))) return rc;
        if ((rc = ensure(h, h->ent_tmp, sizeof(Entry) * (size_t)nbe, true))) return rc;
        if ((rc = ensure(h, h->nv_flags, (size_t)nbe, true))) return rc;
        if ((rc = ensure(h, h->nv_tex, sizeof(uint64_t) * (size_t)((nbe + BSCAN_TILE - 1) / BSCAN_TILE), true)))
            return rc;
        k_nv_claim<<<grid_for(h, nbe), 256, 0, st>>>(it, nbe, h->dense.as<int32_t>(), h->touched.as<int32_t>(), dc);
        NvCounters *hd = static_cast<NvCounters *>(h->hstat);
        cudaMemcpyAsync(hd, dc, sizeof(NvCounters), cudaMemcpyDeviceToHost, st);
        if ((rc = cuda_check(h, cudaStreamSynchronize(st), "node view ids"))) return rc;
        const int64_t n_ids = (int64_t)hd->n_dense;
        uint32_t *kb[2] = {h->sk32[0].as<uint32_t>(), h->sk32[1].as<uint32_t>()};
        uint32_t *vb[2] = {h->sv[0].as<uint32_t>(), h->sv[1].as<uint32_t>()};
        int launches = 0;
        // the ids the first histogram pass notes go to the second key buffer,
        // which the first scatter pass reads and the second one overwrites
        const DenseLoader dl{it, h->dense.as<int32_t>(), kb[1]};
        const NotedIdLoader nl{kb[1]};
        rep.ids = n_ids;
        rep.runs = n_ids;  // one run per distinct node of the batch
        rep.passes = (bits_for((uint64_t)(n_ids > 0 ? n_ids - 1 : 0)) + RADIX_BITS - 1) / RADIX_BITS;
        int r = radix_sort_launch<uint32_t>(dl, nl, nbe, bits_for((uint64_t)(n_ids > 0 ? n_ids - 1 : 0)), kb, vb,
                                            h->hist.as<uint32_t>(), st, &launches);
        if (r < 0) {  // a single distinct node (id 0): the batch order is already grouped
            cudaMemsetAsync(kb[0], 0, sizeof(uint32_t) * (size_t)nbe, st);
            k_iota<<<grid_for(h, nbe), 256, 0, st>>>(vb[0], nbe);
            r = 0;
        }
        // the ids live in the sorted keys and touched[] from here on (the
        // first pass, the id table's only reader, is queued before): clear
        // dense[], with no exit of this call between the claims and here
        k_nv_dense_reset<<<grid_for(h, n_ids), 256, 0, st>>>(h->touched.as<int32_t>(), dc, h->dense.as<int32_t>());
        stage.next("node view: runs and regions");
        uint64_t *part = h->partials.as<uint64_t>();
        // the entries in sorted order, packed once (the runs and the scatter
        // read them coalesced)
        Entry *E = h->ent_tmp.as<Entry>();
        uint8_t *rflags = h->nv_flags.as<uint8_t>();
        k_nv_entries_runs<<<grid_for(h, nbe), 256, 0, st>>>(vb[r], kb[r], it, nbe, slot_base(h, new_lo),
                                                            h->touched.as<int32_t>(), h->ngr.as<NodeRange>(), E,
                                                            rflags);
        AppendRunBytes op{rflags, nbe, kb[r], h->touched.as<int32_t>(), h->run_node.as<int32_t>(),
                          h->run_pos.as<int32_t>(), h->run_g.as<int32_t>(), h->nv_tex.as<uint64_t>()};
        const int nb = bscan_launch(op, part, st);
        // keep the run totals apart: the next scans reuse the partials
        uint64_t *tot = part + SCAN_MAX_BLOCKS + 1;
        cudaMemcpyAsync(tot, part + nb, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
        k_nv_tail<<<1, 1, 0, st>>>(h->run_pos.as<int32_t>(), h->run_g.as<int32_t>(), nullptr, tot, nbe);
        k_nv_reserve<<<grid_for(h, runs_max), 256, 0, st>>>(
            h->run_node.as<int32_t>(), h->run_pos.as<int32_t>(), h->run_g.as<int32_t>(), tot, h->nv_shift, h->e_cap,
            h->g_cap, h->nrec.as<int4>(), h->ngr.as<NodeRange>(), h->nbeg.as<int2>(), h->ngo.as<int32_t>(),
            h->act.as<int32_t>(), h->nrec_n, h->reloc.as<Reloc>(), h->run_de.as<int32_t>(), h->run_dg.as<int32_t>(),
            h->nv_mir.as<NvMirror>(), h->mirror_min, dc);
        h->pending_launches += launches + 6;
        // moves and scatter are queued without a round trip: they read the
        // move count on the device and do nothing when a pool overflowed
        // (the host sees that at the end and rebuilds the view)
        stage.next("node view: region moves and scatter");
        {
            RelocChunkOp rop{h->reloc.as<Reloc>(), h->nv_tmp.as<int32_t>(), dc};
            const int nb2 = scan_launch(rop, n_ids, part, st);  // at most one move per node run
            const int64_t nch_max = (2 * h->e_cap) / RELOC_CHUNK + n_ids;  // bound for the grid only
            int64_t grid = (nch_max + 7) / 8;
            const int64_t gcap = (int64_t)h->num_sms * 16;
            if (grid > gcap) grid = gcap;
            k_nv_reloc<<<(unsigned)grid, 256, 0, st>>>(h->reloc.as<Reloc>(), h->nv_tmp.as<int32_t>(), dc,
                                                       part + nb2, h->ent.as<Entry>(), h->ngo.as<int32_t>(),
                                                       h->ngts.as<int64_t>(),
                                                       h->w_on && h->w_valid && h->gw.p ? h->gw.as<double>() : nullptr);
            h->pending_launches += 4;
        }
        k_nv_scatter<<<(unsigned)(op.tiles() * SCATTER_SPLIT), BSCAN_THREADS, 0, st>>>(
            E, rflags, nbe, h->nv_tex.as<uint64_t>(), h->run_pos.as<int32_t>(), h->run_g.as<int32_t>(),
            h->run_de.as<int32_t>(), h->run_dg.as<int32_t>(), h->run_node.as<int32_t>(), h->e_cap, h->g_cap,
            h->ent.as<Entry>(), h->ngo.as<int32_t>(), h->ngts.as<int64_t>(), h->ngr.as<NodeRange>(), dc);
        h->pending_launches++;
        if ((rc = nv_append_weights(h, nbe))) return rc;
    }
    return cuda_check(h, cudaGetLastError(), "node view append");
}

int nv_append_finish(tempest_t *h, const NvCounters *hc, bool *rebuild)
{
    *rebuild = false;
    NvBatchReport &rep = h->nv_rep;
    const int directed = h->directed;
    if (hc->status)
        return fail(h, TEMPEST_ECUDA, "node view: consistency check failed (code 0x%llx)",
                    (unsigned long long)hc->status);
    if (hc->overflow) {
        *rebuild = true;  // nothing was moved or scattered; the caller rebuilds the whole view
        return TEMPEST_OK;
    }
    if (rep.ev_scanned && (int64_t)hc->ev_removed != rep.ev_entries)
        return fail(h, TEMPEST_ECUDA, "node view: the eviction search removed %lld entries, %lld were evicted",
                    (long long)hc->ev_removed, (long long)rep.ev_entries);
    h->Gn += (int64_t)hc->gn_delta;
    rep.ev_nodes = (int64_t)hc->n_ev_nodes;
    rep.moved_e = (int64_t)hc->moved_e;
    rep.moved_g = (int64_t)hc->moved_g;
    rep.g_added = (int64_t)hc->g_added;
    if (hc->w_rebase) h->w_valid = false;  // a weight exponent grew large: move every reference
    // a node moved onto its copy made ahead: group weights copied before their
    // group grew are stale
    if (hc->mir_switched) h->w_valid = false;
    rep.copied_ahead = (int64_t)hc->mir_switched;
    h->n_act = (int64_t)hc->n_act;
    h->S = h->n_act;
    h->M = directed ? (h->s_hi - h->s_lo) : 2 * (h->s_hi - h->s_lo);
    return TEMPEST_OK;
}

// Canonical arrays of the view (device destination): node segment starts
// (NODE_OFF, N + 1), node order as store positions (M), group starts as
// canonical offsets (Gn + 1), per-node first group (N + 1).
int nv_export(tempest_t *h, int which, int32_t *out)
{
    cudaStream_t st = h->stream;
    const int64_t N = h->N;
    int rc;
    if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
    uint64_t *part = h->partials.as<uint64_t>();
    const int4 *nrec = h->nrec.as<int4>();
    const NodeRange *ngr = h->ngr.as<NodeRange>();
    if (which == TEMPEST_STATE_NODE_OFF || which == TEMPEST_STATE_NODE_GIDX) {
        CountOp op{nrec, ngr, N, which == TEMPEST_STATE_NODE_GIDX, out};
        scan_launch(op, N + 1, part, st);
        return cuda_check(h, cudaGetLastError(), "export");
    }
    // temporaries: canonical segment starts and first groups
    if ((rc = ensure(h, h->nv_tmp, sizeof(int32_t) * 2 * (size_t)(N + 1), true))) return rc;
    int32_t *off = h->nv_tmp.as<int32_t>();
    int32_t *gidx = off + (N + 1);
    CountOp o1{nrec, ngr, N, 0, off};
    scan_launch(o1, N + 1, part, st);
    const int groups = which == TEMPEST_STATE_NODE_GROUP_OFF;
    if (groups) {
        CountOp o2{nrec, ngr, N, 1, gidx};
        scan_launch(o2, N + 1, part, st);
    }
    if (N > 0)
        k_nv_export<<<grid_for(h, 32 * N), 256, 0, st>>>(nrec, ngr, off, gidx, h->ent.as<Entry>(),
                                                         h->ngo.as<int32_t>(), N, slot_base(h, h->s_lo), groups,
                                                         out);
    if (groups) {
        const int32_t Mv = (int32_t)h->M;
        cudaMemcpyAsync(out + h->Gn, &Mv, sizeof(int32_t), cudaMemcpyHostToDevice, st);
    }
    return cuda_check(h, cudaStreamSynchronize(st), "export");
}

}  // namespace tw
