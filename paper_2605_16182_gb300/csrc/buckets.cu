// buckets.cu -- time-bucket tables over the group timestamps of high-degree
// nodes: an index for the first step of every hop, finding the start of
// Gamma_t(v) among v's timestamp groups (Sec. 2.3, 2.5).
//
// A node with G >= BKT_MIN_G groups gets buckets of 2^s time units aligned on
// absolute time (about G >> bkt_log of them over its live range) and a table
// holding, per bucket, the first group whose bucket is at or after it (see
// bkt_rel).  A hop at such a node reads the node's record, one pair of
// adjacent table entries and then bisects the few groups of one bucket,
// instead of bisecting all G groups with one dependent load per level.
//
// The tables depend only on the node view, so they are built once per index
// state, at the first walk call after an ingest, and each build starts from
// the previous one: with buckets on absolute time and groups only appended
// at a node's end or evicted at its front (node-view moves shift a node's
// group indices by one offset, tracked through the groups it has lost), a
// bucket the previous table covers keeps its entry up to that shift, so only
// the buckets of groups appended since are filled from the groups (a node
// whose width drifts more than 4x from its target, or any node after the
// node view was rebuilt, is filled whole):
//   1. a compaction over the nodes that own index regions lists the big
//      nodes, plans each table (width, buckets to copy, groups to scan) and
//      places the tables back to back, each after a small header the next
//      build reads;
//   2. a scan over that list numbers their tasks (copy tasks of BKT_COPY
//      entries, group chunks of BKT_CHUNK groups), and a map gives every task
//      its big node;
//   3. one warp per task copies entries, or reads a chunk's group
//      timestamps, 128 consecutive groups per round, four per lane: group g owns
//      the entries k in (bucket(g - 1), bucket(g)] (it is the first group of
//      those buckets) and the node's last group also (bucket(g), K] (value
//      g1).  The round's buckets go to shared memory and each lane finds the
//      group of one entry by bisecting them, so a round's entries leave as
//      consecutive stores, 32 per store.  Every entry is written once.
#include <algorithm>
#include <climits>

#include "engine.cuh"
#include "prims.cuh"
#include "sortscan.cuh"
#include "walkcore.cuh"

namespace tw {

namespace {

constexpr int32_t BKT_COPY = 2048;   // table entries per copy task

// How a big node's table is built: the bucket width, and which part comes
// from the previous build's table of the node (the buckets both tables cover,
// entries shifted by the node's group renumbering delta) and which part from
// the node's groups (those appended since: from .. g_hi).
struct BktPlan {
    int s;            // log2 of the bucket width
    int64_t bfirst;   // absolute bucket of the node's first live group
    int32_t K;        // buckets
    int32_t ncopy;    // buckets [0, ncopy) copied
    int32_t src;      // previous table's entry for bucket 0, when ncopy > 0
    int32_t delta;    // group index now minus group index then
    int32_t from;     // first group whose buckets are filled from the groups
    int32_t gbase;    // g_lo - groups evicted so far: the group numbering's origin
};

struct BuildCtx {
    const int32_t *prev;  // previous build's tables (null: none usable)
    int prev_gen;         // their generation
    int log_b;
    const int32_t *nev;
};

// Header of a node's table (BKT_HDR int32 before its entries), read by the
// next build: node, generation, width, g_hi and group origin at build time,
// first bucket (two words), buckets.
__device__ __forceinline__ BktPlan bkt_plan(int32_t v, const NodeRange &r, const BuildCtx &bc)
{
    BktPlan p;
    const int32_t G = r.g_hi - r.g_lo;
    const uint64_t span = (uint64_t)r.t_last - (uint64_t)r.t_first;  // >= 1: distinct group timestamps
    const uint64_t kt = (uint64_t)max(1, G >> bc.log_b);
    const uint64_t q = span / kt;
    const int s_fresh = q == 0 ? 0 : 64 - __clzll((long long)q);  // span >> s < kt
    p.gbase = r.g_lo - __ldg(bc.nev + v);
    p.ncopy = 0;
    p.src = -1;
    p.delta = 0;
    p.from = r.g_lo;
    p.s = s_fresh;
    bool reuse = false;
    int64_t old_bfirst = 0;
    int32_t old_K = 0, old_ghi = 0;
    if (bc.prev && (r.bs >> 6) == (bc.prev_gen & 0x3ffffff) && r.tb >= BKT_HDR) {
        const int32_t *hd = bc.prev + r.tb - BKT_HDR;
        const int old_s = hd[2];
        if (hd[0] == v && hd[1] == bc.prev_gen && old_s >= s_fresh - 2 && old_s <= s_fresh + 2) {
            reuse = true;
            p.s = old_s;
            old_ghi = hd[3];
            p.delta = p.gbase - hd[4];
            old_bfirst = (int64_t)(((uint64_t)(uint32_t)hd[6] << 32) | (uint32_t)hd[5]);
            old_K = hd[7];
        }
    }
    p.bfirst = r.t_first >> p.s;
    p.K = (int32_t)((r.t_last >> p.s) - p.bfirst + 1);
    if (reuse) {
        // the live groups' first bucket only moves forward (eviction); the
        // buckets up to the old last one keep their first group
        const int64_t old_blast = old_bfirst + old_K - 1;
        const int64_t nc = min(old_blast, p.bfirst + p.K - 1) - p.bfirst + 1;
        if (p.bfirst >= old_bfirst && nc > 0) {
            p.ncopy = (int32_t)nc;
            p.src = r.tb + (int32_t)(p.bfirst - old_bfirst);
        }
        p.from = max(r.g_lo, old_ghi + p.delta);
        if (p.ncopy == 0) p.from = r.g_lo;
    }
    return p;
}

struct BigNodeOp {
    const int32_t *act;
    NodeRange *ngr;
    BuildCtx bc;
    int gen;
    int32_t *big_node, *big_t;
    int4 *aux0, *aux1;
    int64_t *bf;
    __device__ __forceinline__ uint64_t value(int64_t j) const
    {
        const int32_t v = act[j];
        const NodeRange r = ngr[v];
        if (r.g_hi - r.g_lo < BKT_MIN_G) return 0;
        const BktPlan p = bkt_plan(v, r, bc);
        return (1ull << 32) | (uint64_t)(BKT_HDR + p.K + 1);
    }
    __device__ __forceinline__ void emit(int64_t j, uint64_t x, uint64_t ex) const
    {
        if (!x) return;
        const uint32_t b = (uint32_t)(ex >> 32);
        const int32_t v = act[j];
        const NodeRange r = ngr[v];
        const BktPlan p = bkt_plan(v, r, bc);
        const int32_t base = (int32_t)(uint32_t)ex;
        big_node[b] = v;
        big_t[b] = base;
        aux0[b] = make_int4(p.s, p.from, p.ncopy, p.src);
        aux1[b] = make_int4(p.delta, p.K, (p.ncopy + BKT_COPY - 1) / BKT_COPY, p.gbase);
        bf[b] = p.bfirst;
        ngr[v].tb = base + BKT_HDR;
        ngr[v].bs = ((gen & 0x3ffffff) << 6) | p.s;
    }
};

// Tasks of each big node, over a bound on the big nodes (their count is the
// high half of the big-node scan's total, read on the device: no host round
// trip between the two scans).
struct ChunkOp {
    const int32_t *big_node;
    const NodeRange *ngr;
    const int4 *aux0, *aux1;
    int32_t *big_c;
    const uint64_t *big_tot;
    __device__ __forceinline__ uint64_t value(int64_t b) const
    {
        if (b >= (int64_t)(*big_tot >> 32)) return 0;
        const int4 a0 = aux0[b], a1 = aux1[b];
        const int32_t g_hi = ngr[big_node[b]].g_hi;
        return (uint64_t)a1.z + (uint64_t)((g_hi - a0.y + BKT_CHUNK - 1) / BKT_CHUNK);
    }
    __device__ __forceinline__ void emit(int64_t b, uint64_t, uint64_t ex) const { big_c[b] = (int32_t)ex; }
};

// The big node owning each fill chunk (one warp per big node writes its
// chunk range): the fill then finds a chunk's node with one load.
__global__ void __launch_bounds__(256) k_bkt_owner(const int32_t *__restrict__ big_c, const uint64_t *big_tot,
                                                   int64_t cap_tab, const uint64_t *__restrict__ tot, int64_t cap_ch,
                                                   int32_t *owner, WalkCounters *chk)
{
    const int lane = threadIdx.x & 31;
    const int64_t nb = (int64_t)(*big_tot >> 32);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (int64_t)(uint32_t)*big_tot > cap_tab)
        atomicOr(&chk->status, 1ull << 14);  // tables above their allocated bound (the fill skips them)
    const int64_t nch = (int64_t)*tot;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += warps) {
        const int64_t c0 = __ldg(big_c + b), c1 = b + 1 < nb ? __ldg(big_c + b + 1) : nch;
        if (c1 > cap_ch || c0 > c1) {  // inconsistent lists
            if (lane == 0) atomicOr(&chk->status, 1ull << 13);
            continue;
        }
        for (int64_t c = c0 + lane; c < c1; c += 32) owner[c] = (int32_t)b;
    }
}

// One warp per task (grid-stride, 256-thread blocks).  A node's first tasks
// copy the buckets its previous table already covers (entry + the node's
// renumbering delta, the first clamped to the live groups); the rest fill the
// buckets of its groups from `from` on, a BKT_CHUNK chunk each: entry k, at
// or above the first uncopied bucket, is the first group of bucket >= k (the
// node's last group's buckets after its own hold g_hi).  A node's first task
// writes its header and its entry K.
__global__ void __launch_bounds__(256) k_bkt_fill(const int32_t *__restrict__ big_node,
                                                  const int32_t *__restrict__ big_t,
                                                  const int32_t *__restrict__ big_c,
                                                  const int32_t *__restrict__ owner,
                                                  const int4 *__restrict__ aux0, const int4 *__restrict__ aux1,
                                                  const int64_t *__restrict__ bfs, const uint64_t *__restrict__ tot,
                                                  const NodeRange *__restrict__ ngr,
                                                  const int64_t *__restrict__ ngts, const int32_t *__restrict__ prev,
                                                  int gen, int64_t cap, int32_t *bkt, WalkCounters *chk)
{
    __shared__ __align__(16) int32_t s_bkt[8][128];  // per warp: a round's group buckets
    const int lane = threadIdx.x & 31;
    const int64_t nch = (int64_t)*tot;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += warps) {
        const int64_t b = __ldg(owner + c);
        const int32_t node = __ldg(big_node + b);
        const int32_t g0 = ngr[node].g_lo, g1 = ngr[node].g_hi;
        const int4 a0 = __ldg(aux0 + b), a1 = __ldg(aux1 + b);
        const int s = a0.x, from = a0.y, ncopy = a0.z, src = a0.w;
        const int32_t delta = a1.x, K = a1.y, copy_tasks = a1.z;
        const int64_t bfirst = __ldg(bfs + b);
        const int64_t hb = __ldg(big_t + b);  // header
        const int64_t tb = hb + BKT_HDR;       // entry 0
        const int32_t local = (int32_t)(c - __ldg(big_c + b));
        if (tb + K >= cap || g1 - g0 < BKT_MIN_G || K < 1 || ncopy > K || (ncopy > 0 && !prev)) {
            if (lane == 0) atomicOr(&chk->status, 1ull << 12);  // inconsistent lists
            continue;
        }
        if (local == 0 && lane < BKT_HDR + 1) {
            // header (for the next build) and the end entry
            const int32_t hv[BKT_HDR] = {node, gen, s, g1, a1.w, (int32_t)(uint32_t)bfirst,
                                         (int32_t)(uint32_t)((uint64_t)bfirst >> 32), K};
            if (lane < BKT_HDR) bkt[hb + lane] = hv[lane];
            else bkt[tb + K] = g1;
        }
        if (local < copy_tasks) {
            // eight loads in flight per lane before their stores (the table
            // stores could alias the loads for all the compiler knows)
            const int32_t e0 = local * BKT_COPY, e1 = min(ncopy, e0 + BKT_COPY);
            for (int32_t e = e0 + lane; e < e1; e += 32 * 8) {
                int32_t x[8];
#pragma unroll
                for (int j = 0; j < 8; j++) x[j] = e + 32 * j < e1 ? __ldg(prev + src + e + 32 * j) : 0;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (e + 32 * j < e1) bkt[tb + e + 32 * j] = min(max(x[j] + delta, g0), g1);
            }
            continue;
        }
        const int32_t start = from + (local - copy_tasks) * BKT_CHUNK;
        const int32_t end = min(g1, start + BKT_CHUNK);
        // Rounds of 128 consecutive groups from the 4-aligned group at or
        // before start, four per lane (two 16-byte loads; the next round's in
        // flight), their buckets staged in shared memory.  Buckets are
        // monotone in the group, so entry k (first group of bucket >= k) is
        // found by each lane for its own k by bisecting the round's 128
        // buckets, and a round's entries (the buckets after the last one
        // written, up to its last group's) leave as consecutive stores: about
        // 128 >> log_b of them per round, instead of each group writing its
        // own run.  Groups before the node's first are masked; the node's
        // other groups before start only bound the first entry (carry: the
        // bucket of the group before start, -1 at the node's first group).
        int32_t *sb = s_bkt[threadIdx.x >> 5];
        const int32_t ga = start & ~3;
        int32_t carry = (start > g0 && ga == start) ? (int32_t)((__ldg(ngts + start - 1) >> s) - bfirst) : -1;
        auto load4 = [&](int32_t q, int64_t *t) {
            if (q + 4 <= end) {
                const longlong2 *p2 = reinterpret_cast<const longlong2 *>(ngts + q);
                const longlong2 x = __ldg(p2), y = __ldg(p2 + 1);
                t[0] = x.x;
                t[1] = x.y;
                t[2] = y.x;
                t[3] = y.y;
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) t[j] = q + j < end ? __ldg(ngts + q + j) : 0;
            }
        };
        int64_t tv[4];
        load4(ga + 4 * lane, tv);
        for (int32_t gb = ga; gb < end; gb += 128) {
            const int32_t q = gb + 4 * lane;
            int64_t tn[4];
            load4(q + 128, tn);
            int4 kq;
            kq.x = q < g0 ? INT_MIN : (int32_t)((tv[0] >> s) - bfirst);
            kq.y = q + 1 < g0 ? INT_MIN : (int32_t)((tv[1] >> s) - bfirst);
            kq.z = q + 2 < g0 ? INT_MIN : (int32_t)((tv[2] >> s) - bfirst);
            kq.w = q + 3 < g0 ? INT_MIN : (int32_t)((tv[3] >> s) - bfirst);
            __syncwarp();
            reinterpret_cast<int4 *>(sb)[lane] = kq;
            __syncwarp();
            const int32_t last = min(end, gb + 128) - 1 - gb;  // the round's last group (index in the round)
            if (gb == ga && start > g0 && ga < start) carry = sb[start - 1 - ga];
            const int32_t hi = sb[last];
            // the node's last group also owns the buckets after its own, up to K
            const int32_t top = gb + last == g1 - 1 ? K : hi;
            for (int32_t kb = max(carry + 1, ncopy); kb <= top; kb += 32) {
                const int32_t k = kb + lane;
                if (k <= top) {
                    int32_t v = g1;
                    if (k <= hi) {
                        int32_t lo = 0, up = last;  // sb[last] = hi >= k
                        while (lo < up) {
                            const int32_t mid = (lo + up) >> 1;
                            if (sb[mid] >= k) up = mid;
                            else lo = mid + 1;
                        }
                        v = gb + lo;
                    }
                    bkt[tb + k] = v;
                }
            }
            carry = hi;
#pragma unroll
            for (int j = 0; j < 4; j++) tv[j] = tn[j];
        }
    }
}

// Active nodes (at least one live group) in id order.
struct ActiveOp {
    const NodeRange *ngr;
    int64_t N;
    int32_t *out;
    __device__ __forceinline__ uint64_t value(int64_t v) const
    {
        return v < N && ngr[v].g_hi > ngr[v].g_lo ? 1u : 0u;
    }
    __device__ __forceinline__ void emit(int64_t v, uint64_t x, uint64_t ex) const
    {
        if (x) out[ex] = (int32_t)v;
    }
};

}  // namespace

int prepare_active_nodes(tempest_t *h)
{
    int rc;
    if ((rc = views_repair(h))) return rc;
    if (h->pn_ver == h->state_ver) return TEMPEST_OK;
    const int64_t N = h->N;
    h->n_pn = 0;
    if (N > 0 && h->nv_ready && h->M > 0) {
        if ((rc = ensure(h, h->pn_nodes, sizeof(int32_t) * (size_t)N, true))) return rc;
        if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
        ActiveOp op{h->ngr.as<NodeRange>(), N, h->pn_nodes.as<int32_t>()};
        const int nb = scan_launch(op, N, h->partials.as<uint64_t>(), h->stream);
        uint64_t *hp = static_cast<uint64_t *>(h->hstat);
        cudaMemcpyAsync(hp, h->partials.as<uint64_t>() + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream);
        if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "active nodes"))) return rc;
        h->n_pn = (int64_t)hp[0];
    }
    h->pn_ver = h->state_ver;
    return TEMPEST_OK;
}

int prepare_walk_index(tempest_t *h)
{
    int rc;
    if ((rc = views_repair(h))) return rc;
    if (h->bkt_ver == h->state_ver) return TEMPEST_OK;
    cudaStream_t st = h->stream;
    const int64_t S = h->n_act, Gn = h->Gn;
    h->n_big = 0;
    if (S > 0 && Gn >= BKT_MIN_G) {
        const size_t Sz = (size_t)S;
        if ((rc = ensure(h, h->big_node, sizeof(int32_t) * Sz, true))) return rc;
        if ((rc = ensure(h, h->big_t, sizeof(int32_t) * Sz, true))) return rc;
        if ((rc = ensure(h, h->big_c, sizeof(int32_t) * Sz, true))) return rc;
        if ((rc = ensure(h, h->big_aux0, sizeof(int4) * Sz, true))) return rc;
        if ((rc = ensure(h, h->big_aux1, sizeof(int4) * Sz, true))) return rc;
        if ((rc = ensure(h, h->big_bf, sizeof(int64_t) * Sz, true))) return rc;
        if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
        if ((rc = ensure(h, h->wcnt, sizeof(WalkCounters)))) return rc;
        // the previous build's tables become the copy source; the new ones
        // go to the other buffer, sized for the most a build can need: a
        // width within 4x of its target gives K <= 4 max(1, G >> log_b) + 1,
        // so a node takes at most 4 (G >> log_b) + 14 with its header and end
        std::swap(h->bkt, h->bkt_prev);
        const bool prev_ok = h->bkt_prev_ok && h->bkt_prev.p != nullptr;
        const int prev_gen = h->bkt_gen;
        const int gen = ++h->bkt_gen;
        h->bkt_prev_ok = false;
        const int64_t bound = 4 * (Gn >> h->bkt_log) + 16 * (Gn / BKT_MIN_G + 1) + 64;
        if (bound >= (int64_t)INT32_MAX)
            return fail(h, TEMPEST_ENOMEM, "walk index: %lld bucket entries exceed the int32 range",
                        (long long)bound);
        if ((rc = ensure(h, h->bkt, sizeof(int32_t) * (size_t)bound, true))) return rc;
        uint64_t *part = h->partials.as<uint64_t>();
        NodeRange *ngr = h->ngr.as<NodeRange>();
        const BuildCtx bc{prev_ok ? h->bkt_prev.as<int32_t>() : nullptr, prev_gen, h->bkt_log, h->nev.as<int32_t>()};
        BigNodeOp op{h->act.as<int32_t>(), ngr, bc, gen, h->big_node.as<int32_t>(), h->big_t.as<int32_t>(),
                     h->big_aux0.as<int4>(), h->big_aux1.as<int4>(), h->big_bf.as<int64_t>()};
        const int nblk = scan_launch<BigNodeOp, 1>(op, S, part, st);
        // the big-node count and table size stay on the device (kept apart:
        // the next scan reuses the partials); sizes below use host bounds
        uint64_t *big_tot = part + SCAN_MAX_BLOCKS + 1;
        cudaMemcpyAsync(big_tot, part + nblk, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
        ChunkOp cop{h->big_node.as<int32_t>(), ngr, h->big_aux0.as<int4>(), h->big_aux1.as<int4>(),
                    h->big_c.as<int32_t>(), big_tot};
        const int nblk2 = scan_launch<ChunkOp, 1>(cop, S, part, st);
        // the fill's consistency flag goes to the walk counters, which
        // every walk call zeroes before its kernels: read it here
        cudaMemsetAsync(h->wcnt.p, 0, sizeof(WalkCounters), st);
        // tasks <= copy tasks + group chunks <= bound / BKT_COPY + Gn / BKT_CHUNK + 2 S
        const int64_t nch_max = bound / BKT_COPY + Gn / BKT_CHUNK + 2 * S + 1;
        if ((rc = ensure(h, h->big_own, sizeof(int32_t) * (size_t)nch_max, true))) return rc;
        const int64_t gcap = (int64_t)h->num_sms * 16;
        int64_t ogrid = (S + 7) / 8;
        if (ogrid > gcap) ogrid = gcap;
        k_bkt_owner<<<(unsigned)ogrid, 256, 0, st>>>(h->big_c.as<int32_t>(), big_tot, bound, part + nblk2, nch_max,
                                                     h->big_own.as<int32_t>(), h->wcnt.as<WalkCounters>());
        int64_t grid = (nch_max + 7) / 8;
        if (grid > gcap) grid = gcap;
        k_bkt_fill<<<(unsigned)grid, 256, 0, st>>>(
            h->big_node.as<int32_t>(), h->big_t.as<int32_t>(), h->big_c.as<int32_t>(), h->big_own.as<int32_t>(),
            h->big_aux0.as<int4>(), h->big_aux1.as<int4>(), h->big_bf.as<int64_t>(), part + nblk2, ngr,
            h->ngts.as<int64_t>(), bc.prev, gen, bound, h->bkt.as<int32_t>(), h->wcnt.as<WalkCounters>());
        WalkCounters *hc = static_cast<WalkCounters *>(h->hstat);
        uint64_t *hb = reinterpret_cast<uint64_t *>(static_cast<char *>(h->hstat) + 2048);
        cudaMemcpyAsync(hc, h->wcnt.p, sizeof(WalkCounters), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(hb, big_tot, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
        if ((rc = cuda_check(h, cudaStreamSynchronize(st), "bucket fill"))) return rc;
        if (hc->status)
            return fail(h, TEMPEST_ECUDA, "walk index: bucket table check failed (code 0x%llx)",
                        (unsigned long long)hc->status);
        const int64_t nb = (int64_t)(hb[0] >> 32);
        h->n_big = nb;
        h->bkt_prev_ok = true;  // these tables are the next build's source
    }
    h->bkt_ver = h->state_ver;
    return TEMPEST_OK;
}

}  // namespace tw
