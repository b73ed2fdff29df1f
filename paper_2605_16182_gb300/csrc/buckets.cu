// buckets.cu -- time-bucket tables over the group timestamps of high-degree
// nodes: an index for the first step of every hop, finding the start of
// Gamma_t(v) among v's timestamp groups (Sec. 2.3, 2.5).
//
// A node with G >= BKT_MIN_G groups gets K = G >> bkt_log buckets over its
// timestamp range and a table of K + 1 group indices (see bkt_map).  A hop at
// such a node reads the node's first and last group timestamps, one pair of
// adjacent table entries and then bisects the few groups of one bucket,
// instead of bisecting all G groups with one dependent load per level.
//
// The tables depend only on the node view, so they are built once per index
// state, at the first walk call after an ingest:
//   1. a compaction over the nodes that own index regions lists the big
//      nodes and places their tables back to back (prefix of K + 1);
//   2. a scan over that list numbers their fill chunks (BKT_CHUNK groups),
//      and a map gives every chunk its big node;
//   3. one warp per chunk reads the chunk's group timestamps, each lane 32
//      consecutive groups in order (one cached load per group);
//      group g owns the table entries k in (bucket(g - 1), bucket(g)] (it is
//      the first group of those buckets) and the node's last group also
//      owns (bucket(g), K] (value g1).  A group's lane writes its own few
//      entries; a long run (a time gap that leaves many buckets empty) is
//      written by the whole warp, 32 entries per store instruction rather
//      than by one lane.  Every entry is written once.
#include "engine.cuh"
#include "prims.cuh"
#include "walkcore.cuh"

namespace tw {

namespace {

constexpr int BKT_SHORT_RUN = 4;  // table entries a group's own lane writes

struct BigNodeOp {
    const int32_t *act;
    NodeRange *ngr;
    int log_b;
    int32_t *big_node, *big_t;
    __device__ __forceinline__ uint64_t value(int64_t j) const
    {
        const NodeRange &r = ngr[act[j]];
        const int32_t G = r.g_hi - r.g_lo;
        if (G < BKT_MIN_G) return 0;
        return (1ull << 32) | (uint64_t)(bkt_count(G, log_b) + 1u);
    }
    __device__ __forceinline__ void emit(int64_t j, uint64_t v, uint64_t ex) const
    {
        if (!v) return;
        const uint32_t b = (uint32_t)(ex >> 32);
        const int32_t node = act[j];
        big_node[b] = node;
        big_t[b] = (int32_t)(uint32_t)ex;
        ngr[node].tb = (int32_t)(uint32_t)ex;
    }
};

struct ChunkOp {
    const int32_t *big_node;
    const NodeRange *ngr;
    int32_t *big_c;
    __device__ __forceinline__ uint64_t value(int64_t b) const
    {
        const NodeRange &r = ngr[big_node[b]];
        return (uint64_t)((r.g_hi - r.g_lo + BKT_CHUNK - 1) / BKT_CHUNK);
    }
    __device__ __forceinline__ void emit(int64_t b, uint64_t, uint64_t ex) const { big_c[b] = (int32_t)ex; }
};

// The big node owning each fill chunk (one warp per big node writes its
// chunk range): the fill then finds a chunk's node with one load.
__global__ void __launch_bounds__(256) k_bkt_owner(const int32_t *__restrict__ big_c, int64_t nb,
                                                   const uint64_t *__restrict__ tot, int64_t cap_ch,
                                                   int32_t *owner, WalkCounters *chk)
{
    const int lane = threadIdx.x & 31;
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

// One warp per chunk of BKT_CHUNK groups (grid-stride); lane i takes the
// chunk's groups [32 i, 32 i + 32) in order, so a group costs one cached load
// and a few instructions; totals of the compaction in tot.
__global__ void __launch_bounds__(256) k_bkt_fill(const int32_t *__restrict__ big_node,
                                                  const int32_t *__restrict__ big_t,
                                                  const int32_t *__restrict__ big_c,
                                                  const int32_t *__restrict__ owner,
                                                  const uint64_t *__restrict__ tot,
                                                  const NodeRange *__restrict__ ngr,
                                                  const int64_t *__restrict__ ngts, int log_b, int64_t cap,
                                                  int32_t *bkt, WalkCounters *chk)
{
    static_assert(BKT_CHUNK == 32 * 32, "a chunk is 32 groups per lane");
    const int lane = threadIdx.x & 31;
    const int64_t nch = (int64_t)*tot;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += warps) {
        const int64_t b = __ldg(owner + c);
        const int32_t node = __ldg(big_node + b);
        const int32_t g0 = ngr[node].g_lo, g1 = ngr[node].g_hi;
        const uint32_t K = bkt_count(g1 - g0, log_b);
        const int64_t tb = __ldg(big_t + b);
        if (tb + K >= cap || g1 - g0 < BKT_MIN_G) {  // inconsistent lists
            if (lane == 0) atomicOr(&chk->status, 1ull << 12);
            continue;
        }
        const BktMap bm = bkt_map(__ldg(ngts + g0), __ldg(ngts + g1 - 1), K);
        const int32_t start = g0 + (int32_t)(c - __ldg(big_c + b)) * BKT_CHUNK;
        const int32_t end = min(g1, start + BKT_CHUNK);
        const int32_t my0 = start + 32 * lane, my1 = min(end, my0 + 32);
        // bucket of the group before this lane's first (-1 at the node's first group)
        int32_t kp = (my0 == g0 || my0 >= end) ? -1 : (int32_t)bkt_index(bm, __ldg(ngts + my0 - 1));
        // timestamps come in 8 at a time (four 16-byte loads in flight when
        // the lane's groups start 16-byte aligned, else element loads)
        const bool vec = (((uintptr_t)(ngts + my0)) & 15) == 0;
        for (int jb = 0; jb < 32; jb += 8) {
            int64_t tv[8];
            const int32_t gb = my0 + jb;
            if (vec && gb + 8 <= my1) {
                const longlong2 *q = reinterpret_cast<const longlong2 *>(ngts + gb);
#pragma unroll
                for (int x = 0; x < 4; x++) {
                    const longlong2 v2 = __ldg(q + x);
                    tv[2 * x] = v2.x;
                    tv[2 * x + 1] = v2.y;
                }
            } else {
#pragma unroll
                for (int x = 0; x < 8; x++) tv[x] = gb + x < my1 ? __ldg(ngts + gb + x) : 0;
            }
#pragma unroll
            for (int x = 0; x < 8; x++) {
                const int32_t g = gb + x;
                const bool valid = g < my1;
                const int32_t k = valid ? (int32_t)bkt_index(bm, tv[x]) : kp;
                // entries (kp, k] hold g; the last group adds (k, K] holding g1
                const bool last = valid && g == g1 - 1;
                const int32_t lo_k = kp + 1;
                const int32_t cnt = valid ? (last ? (int32_t)K : k) - kp : 0;
                // a short run (the common case: about one bucket per group) is
                // written by its own lane; long runs (time gaps that leave many
                // buckets empty) by the whole warp, 32 entries per store
                if (cnt <= BKT_SHORT_RUN) {
                    for (int32_t e = 0; e < cnt; e++) {
                        const int32_t kk = lo_k + e;
                        bkt[tb + kk] = kk <= k ? g : g1;
                    }
                }
                unsigned longs = __ballot_sync(0xffffffffu, cnt > BKT_SHORT_RUN);
                while (longs) {
                    const int r = __ffs(longs) - 1;
                    longs &= longs - 1;
                    const int32_t r_lo = __shfl_sync(0xffffffffu, lo_k, r);
                    const int32_t r_cnt = __shfl_sync(0xffffffffu, cnt, r);
                    const int32_t r_k = __shfl_sync(0xffffffffu, k, r);
                    const int32_t r_g = __shfl_sync(0xffffffffu, g, r);
                    for (int32_t e = lane; e < r_cnt; e += 32) {
                        const int32_t kk = r_lo + e;
                        bkt[tb + kk] = kk <= r_k ? r_g : g1;
                    }
                }
                kp = k;
            }
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
    if (h->pn_ver == h->state_ver) return TEMPEST_OK;
    const int64_t N = h->N;
    int rc;
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
    if (h->bkt_ver == h->state_ver) return TEMPEST_OK;
    cudaStream_t st = h->stream;
    const int64_t S = h->n_act, Gn = h->Gn;
    int rc;
    h->n_big = 0;
    if (S > 0 && Gn >= BKT_MIN_G) {
        const size_t Sz = (size_t)S;
        if ((rc = ensure(h, h->big_node, sizeof(int32_t) * Sz, true))) return rc;
        if ((rc = ensure(h, h->big_t, sizeof(int32_t) * Sz, true))) return rc;
        if ((rc = ensure(h, h->big_c, sizeof(int32_t) * Sz, true))) return rc;
        if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
        if ((rc = ensure(h, h->wcnt, sizeof(WalkCounters)))) return rc;
        uint64_t *part = h->partials.as<uint64_t>();
        NodeRange *ngr = h->ngr.as<NodeRange>();
        BigNodeOp op{h->act.as<int32_t>(), ngr, h->bkt_log, h->big_node.as<int32_t>(), h->big_t.as<int32_t>()};
        const int nblk = scan_launch(op, S, part, st);
        uint64_t *hp = static_cast<uint64_t *>(h->hstat);
        cudaMemcpyAsync(hp, part + nblk, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
        if ((rc = cuda_check(h, cudaStreamSynchronize(st), "bucket lists"))) return rc;
        const uint64_t tot = hp[0];
        const int64_t nb = (int64_t)(tot >> 32), cap = (int64_t)(uint32_t)tot;
        if (cap >= (int64_t)INT32_MAX)
            return fail(h, TEMPEST_ENOMEM, "walk index: %lld bucket entries exceed the int32 range",
                        (long long)cap);
        if (nb > 0) {
            if ((rc = ensure(h, h->bkt, sizeof(int32_t) * (size_t)cap, true))) return rc;
            ChunkOp cop{h->big_node.as<int32_t>(), ngr, h->big_c.as<int32_t>()};
            const int nblk2 = scan_launch(cop, nb, part, st);
            // the fill's consistency flag goes to the walk counters, which
            // every walk call zeroes before its kernels: read it here
            cudaMemsetAsync(h->wcnt.p, 0, sizeof(WalkCounters), st);
            const int64_t nch_max = Gn / BKT_CHUNK + nb;  // chunks <= sum(G / CHUNK + 1)
            if ((rc = ensure(h, h->big_own, sizeof(int32_t) * (size_t)nch_max, true))) return rc;
            const int64_t gcap = (int64_t)h->num_sms * 16;
            int64_t ogrid = (nb + 7) / 8;
            if (ogrid > gcap) ogrid = gcap;
            k_bkt_owner<<<(unsigned)ogrid, 256, 0, st>>>(h->big_c.as<int32_t>(), nb, part + nblk2, nch_max,
                                                         h->big_own.as<int32_t>(), h->wcnt.as<WalkCounters>());
            int64_t grid = (nch_max + 7) / 8;
            if (grid > gcap) grid = gcap;
            k_bkt_fill<<<(unsigned)grid, 256, 0, st>>>(h->big_node.as<int32_t>(), h->big_t.as<int32_t>(),
                                                       h->big_c.as<int32_t>(), h->big_own.as<int32_t>(),
                                                       part + nblk2, ngr, h->ngts.as<int64_t>(), h->bkt_log, cap,
                                                       h->bkt.as<int32_t>(), h->wcnt.as<WalkCounters>());
            WalkCounters *hc = static_cast<WalkCounters *>(h->hstat);
            cudaMemcpyAsync(hc, h->wcnt.p, sizeof(WalkCounters), cudaMemcpyDeviceToHost, st);
            if ((rc = cuda_check(h, cudaStreamSynchronize(st), "bucket fill"))) return rc;
            if (hc->status)
                return fail(h, TEMPEST_ECUDA, "walk index: bucket table check failed (code 0x%llx)",
                            (unsigned long long)hc->status);
        }
        h->n_big = nb;
    }
    h->bkt_ver = h->state_ver;
    return TEMPEST_OK;
}

}  // namespace tw
