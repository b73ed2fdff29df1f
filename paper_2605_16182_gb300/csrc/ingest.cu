// ingest.cu -- streaming ingestion, window eviction and the dual index
// (Tempest Sec. 2.3 and 2.6).
//
// Per batch:
//   1. one pass over the batch: timestamp range, largest id, negative ids,
//      late edges (older than the cut-off in force), whether it is sorted;
//   2. a stable radix sort of the batch on timestamp (skipped when the batch
//      arrived sorted); late edges are then a prefix and are skipped;
//   3. the new cut-off is found without materialising the merge (a merge-path
//      search gives the timestamp at any rank of the merged order), and the
//      first kept element of the store and of the batch by binary search;
//   4. the kept store suffix and the kept batch are merged into the other
//      store buffer (two copies when the batch starts no earlier than the
//      store ends, a merge-path merge otherwise);
//   5. timestamp-grouped view: compaction of the run starts of equal ts;
//   6. node view: stable radix sort of the store's (node, slot) pairs by
//      node, one 16-byte entry per slot, then one compaction that emits the
//      (node, ts) group starts and the node segment starts, and an exclusive
//      scan of per-node group counts that gives each node's first group.
#include <stdio.h>

#include "engine.cuh"
#include "prims.cuh"

namespace tw {

// ---------------------------------------------------------------------------
// batch statistics
// ---------------------------------------------------------------------------
__global__ void k_batch_stats(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                              const int64_t *__restrict__ ts, int64_t n, int has_cut, long long cut,
                              IngestScratch *o)
{
    long long tmin = LLONG_MAX, tmax = LLONG_MIN;
    int maxid = 0, neg = 0;
    unsigned long long late = 0, uns = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[i], b = dst[i];
        const long long t = ts[i];
        tmin = min(tmin, t);
        tmax = max(tmax, t);
        maxid = max(maxid, max(a, b));
        neg |= (a < 0) | (b < 0);
        late += (has_cut && t < cut) ? 1ull : 0ull;
        if (i > 0 && ts[i - 1] > t) uns++;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, d));
        tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, d));
        maxid = max(maxid, __shfl_xor_sync(0xffffffffu, maxid, d));
        neg |= __shfl_xor_sync(0xffffffffu, neg, d);
        late += __shfl_xor_sync(0xffffffffu, late, d);
        uns += __shfl_xor_sync(0xffffffffu, uns, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&o->ts_min, tmin);
        atomicMax(&o->ts_max, tmax);
        atomicMax(&o->max_id, maxid);
        if (neg) atomicOr(&o->neg_id, 1);
        if (late) atomicAdd(&o->late, late);
        if (uns) atomicAdd(&o->unsorted, uns);
    }
}

__global__ void k_init_scratch(IngestScratch *o)
{
    o->ts_min = LLONG_MAX;
    o->ts_max = LLONG_MIN;
    o->max_id = 0;
    o->neg_id = 0;
    o->late = 0;
    o->unsorted = 0;
    o->cut = 0;
    o->has_cut = 0;
    o->i0 = 0;
    o->j0 = 0;
    o->kept_batch_min_ts = 0;
    o->store_last_ts = 0;
    o->status = 0;
}

struct TsKeyLoader {
    const int64_t *ts;
    long long tmin;
    __device__ __forceinline__ unsigned long long key(int64_t i) const
    {
        return (unsigned long long)ts[i] - (unsigned long long)tmin;
    }
    __device__ __forceinline__ uint32_t val(int64_t i) const { return (uint32_t)i; }
};

__global__ void k_gather_batch(const uint32_t *__restrict__ perm, const int32_t *__restrict__ src,
                               const int32_t *__restrict__ dst, const int64_t *__restrict__ ts, int64_t n,
                               int32_t *osrc, int32_t *odst, int64_t *ots)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = perm[i];
        osrc[i] = src[p];
        odst[i] = dst[p];
        ots[i] = ts[p];
    }
}

// ---------------------------------------------------------------------------
// merge-path helpers.  Merge order: a (the store) before b (the batch) on
// equal timestamps, since every batch edge arrived after every store edge.
// Returns the number of a-elements among the first r merged elements.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t merge_split(const int64_t *a, int64_t na, const int64_t *b, int64_t nb,
                                               int64_t r)
{
    int64_t lo = r > nb ? r - nb : 0;
    int64_t hi = r < na ? r : na;
    while (lo < hi) {
        const int64_t i = lo + ((hi - lo) >> 1);
        const int64_t j = r - i;  // j >= 1 here since i < hi <= r ... when j == 0 the split is found
        // does a[i] come after b[j-1]?
        if (j == 0 || b[j - 1] < a[i]) hi = i;
        else lo = i + 1;
    }
    return lo;
}

__device__ __forceinline__ int64_t lower_bound_i64(const int64_t *a, int64_t n, int64_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One thread: new cut-off and the first kept element of store / batch.
// mode: 0 none, 1 duration (param = Delta), 2 count (param = W).
__global__ void k_window(int mode, long long param, const int64_t *old_ts, int64_t m_old,
                         const int64_t *bts, int64_t nb, int has_old, long long cut_old, IngestScratch *o)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int has = has_old;
    long long cut = cut_old;
    if (mode == 1 && m_old + nb > 0) {
        long long tmax = LLONG_MIN;
        if (m_old > 0) tmax = old_ts[m_old - 1];
        if (nb > 0) tmax = max(tmax, (long long)bts[nb - 1]);
        const long long c = (tmax < LLONG_MIN + param) ? LLONG_MIN : tmax - param;
        if (!has || c > cut) cut = c;
        has = 1;
    } else if (mode == 2 && m_old + nb > param) {
        const int64_t r = m_old + nb - param;  // rank of the W-th newest element
        const int64_t i = merge_split(old_ts, m_old, bts, nb, r);
        const int64_t j = r - i;
        long long c;
        if (j >= nb || (i < m_old && old_ts[i] <= bts[j])) c = old_ts[i];
        else c = bts[j];
        if (!has || c > cut) cut = c;
        has = 1;
    }
    int64_t i0 = 0, j0 = 0;
    if (has) {
        i0 = lower_bound_i64(old_ts, m_old, cut);
        j0 = lower_bound_i64(bts, nb, cut);
    }
    o->cut = cut;
    o->has_cut = has;
    o->i0 = i0;
    o->j0 = j0;
    o->kept_batch_min_ts = (j0 < nb) ? bts[j0] : LLONG_MAX;
    o->store_last_ts = (m_old > 0) ? old_ts[m_old - 1] : LLONG_MIN;
}

// General merge of two (ts)-sorted SoA runs; each thread produces MERGE_K
// consecutive outputs.
constexpr int MERGE_K = 8;
__global__ void k_merge(const int32_t *__restrict__ as, const int32_t *__restrict__ ad,
                        const int64_t *__restrict__ at, int64_t na, const int32_t *__restrict__ bs,
                        const int32_t *__restrict__ bd, const int64_t *__restrict__ bt, int64_t nb,
                        int32_t *os, int32_t *od, int64_t *ot)
{
    const int64_t n = na + nb;
    const int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * MERGE_K;
    if (r0 >= n) return;
    int64_t i = merge_split(at, na, bt, nb, r0);
    int64_t j = r0 - i;
    const int64_t r1 = min(n, r0 + MERGE_K);
    for (int64_t r = r0; r < r1; r++) {
        if (j >= nb || (i < na && at[i] <= bt[j])) {
            os[r] = as[i];
            od[r] = ad[i];
            ot[r] = at[i];
            i++;
        } else {
            os[r] = bs[j];
            od[r] = bd[j];
            ot[r] = bt[j];
            j++;
        }
    }
}

// ---------------------------------------------------------------------------
// views
// ---------------------------------------------------------------------------
struct TsGroupOp {
    const int64_t *ts;
    int32_t *goff;
    __device__ __forceinline__ uint64_t value(int64_t i) const
    {
        return (i == 0 || ts[i] != ts[i - 1]) ? 1u : 0u;
    }
    __device__ __forceinline__ void emit(int64_t i, uint64_t v, uint64_t ex) const
    {
        if (v) goff[ex] = (int32_t)i;
    }
};

struct StoreKeyLoader {
    const int32_t *src, *dst;
    int directed;
    __device__ __forceinline__ uint32_t key(int64_t i) const
    {
        if (directed) return (uint32_t)src[i];
        return (uint32_t)((i & 1) ? dst[i >> 1] : src[i >> 1]);
    }
    __device__ __forceinline__ uint32_t val(int64_t i) const { return (uint32_t)i; }
};

__global__ void k_node_entries(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ slots,
                               const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                               const int64_t *__restrict__ ts, int directed, int64_t M, Entry *E, int32_t *enode)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t slot = slots[i];
        const int64_t pos = directed ? (int64_t)slot : (int64_t)(slot >> 1);
        const bool side = !directed && (slot & 1u);
        Entry e;
        e.ts = ts[pos];
        e.other = side ? src[pos] : dst[pos];
        e.slot = (int32_t)slot;
        E[i] = e;
        enode[i] = (int32_t)keys[i];
    }
}

// Packed counter: high 32 bits count node segments, low 32 bits count
// (node, ts) groups.
struct NodeGroupOp {
    const int32_t *enode;  // node of each entry (entries grouped by node)
    const Entry *E;
    int32_t *ngo;
    int64_t *ngts;
    int32_t *seg_node;
    int32_t *seg_g;
    __device__ __forceinline__ uint64_t value(int64_t i) const
    {
        if (i == 0) return (1ull << 32) | 1ull;
        const bool seg = enode[i] != enode[i - 1];
        const bool grp = seg || E[i].ts != E[i - 1].ts;
        return ((uint64_t)seg << 32) | (uint64_t)grp;
    }
    __device__ __forceinline__ void emit(int64_t i, uint64_t v, uint64_t ex) const
    {
        if (v & 1ull) {
            const uint32_t g = (uint32_t)ex;
            ngo[g] = (int32_t)i;
            ngts[g] = E[i].ts;
            if (v >> 32) {
                const uint32_t j = (uint32_t)(ex >> 32);
                seg_node[j] = enode[i];
                seg_g[j] = (int32_t)g;
            }
        }
    }
};

__global__ void k_seg_counts(const int32_t *__restrict__ seg_node, const int32_t *__restrict__ seg_g,
                             int64_t S, int64_t Gn, int32_t *gcnt)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t next = (j + 1 < S) ? seg_g[j + 1] : Gn;
        gcnt[seg_node[j]] = (int32_t)(next - seg_g[j]);
    }
}

struct GidxOp {
    const int32_t *gcnt;
    int64_t N;
    int32_t *gidx;
    __device__ __forceinline__ uint64_t value(int64_t v) const { return v < N ? (uint64_t)gcnt[v] : 0ull; }
    __device__ __forceinline__ void emit(int64_t v, uint64_t, uint64_t ex) const { gidx[v] = (int32_t)ex; }
};

__global__ void k_set_i32(int32_t *p, int32_t v) { *p = v; }

__global__ void k_node_off(const int32_t *__restrict__ gidx, const int32_t *__restrict__ ngo, int64_t N,
                           int32_t *node_off)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= N;
         v += (int64_t)gridDim.x * blockDim.x)
        node_off[v] = ngo[gidx[v]];
}

__global__ void k_node_order(const Entry *__restrict__ E, int64_t M, int32_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = E[i].slot;
}

// ---- incremental node view (the batch starts no earlier than the store ends)

// Entries of the evicted store prefix [0, i0), counted per node.  Every
// node loses a prefix of its segment: eviction removes the oldest edges.
__global__ void k_evict_counts(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t items,
                               int directed, int64_t N, int32_t *ev, IngestScratch *chk)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < items;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = directed ? src[i] : ((i & 1) ? dst[i >> 1] : src[i >> 1]);
        if (v < 0 || v >= N) {
            atomicOr(&chk->status, 1ull << 0);
            v = -1;
        }
        const unsigned am = __activemask();
        const unsigned peers = __match_any_sync(am, v);
        if (v >= 0 && lane == __ffs(peers) - 1) atomicAdd(&ev[v], __popc(peers));
    }
}

// (node, slot) pairs of the batch's entries, slots numbered in the new store
// where the batch occupies positions [base, base + nb).
struct BatchKeyLoader {
    const int32_t *src, *dst;
    int directed;
    int64_t base;
    __device__ __forceinline__ uint32_t key(int64_t i) const
    {
        if (directed) return (uint32_t)src[base + i];
        return (uint32_t)((i & 1) ? dst[base + (i >> 1)] : src[base + (i >> 1)]);
    }
    __device__ __forceinline__ uint32_t val(int64_t i) const
    {
        return (uint32_t)(directed ? base + i : 2 * base + i);
    }
};

// Runs of equal nodes in the sorted batch keys: bstart[v] = first index,
// bcnt[v] = run length (bcnt starts at 0; pass 0 stores the run end, pass 1
// subtracts the start).
__global__ void k_batch_runs(const uint32_t *__restrict__ K, int64_t n, int pass, int32_t *bstart, int32_t *bcnt)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = K[j];
        if (pass == 0) {
            if (j == 0 || K[j - 1] != v) bstart[v] = (int32_t)j;
            if (j == n - 1 || K[j + 1] != v) bcnt[v] = (int32_t)(j + 1);
        } else if (j == 0 || K[j - 1] != v) {
            bcnt[v] -= (int32_t)j;
        }
    }
}

// New segment starts: kept old entries plus new entries, per node.
struct NoffOp {
    const int32_t *noff_old;
    int64_t N_old;
    const int32_t *ev;
    const int32_t *bcnt;
    int64_t N;
    int32_t *noff_new;
    __device__ __forceinline__ uint64_t value(int64_t v) const
    {
        if (v >= N) return 0;
        const int32_t old = v < N_old ? noff_old[v + 1] - noff_old[v] : 0;
        return (uint64_t)(old - ev[v] + bcnt[v]);
    }
    __device__ __forceinline__ void emit(int64_t v, uint64_t, uint64_t ex) const { noff_new[v] = (int32_t)ex; }
};

// Kept old entries move by a per-node shift; their slots shift by E0 (the
// evicted store prefix, in slots).
__global__ void k_copy_kept(const Entry *__restrict__ E_old, const int32_t *__restrict__ enode_old, int64_t M_old,
                            const int32_t *__restrict__ noff_old, const int32_t *__restrict__ ev,
                            const int32_t *__restrict__ noff_new, int32_t E0, int64_t N_old, int64_t M_new,
                            Entry *E_new, int32_t *enode_new, IngestScratch *chk)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M_old;
         i += (int64_t)gridDim.x * blockDim.x) {
        Entry e = E_old[i];
        if (e.slot < E0) continue;  // evicted
        const int32_t v = enode_old[i];
        if (v < 0 || v >= N_old) {
            atomicOr(&chk->status, 1ull << 1);
            continue;
        }
        const int64_t p = (int64_t)noff_new[v] + (i - noff_old[v] - ev[v]);
        if (p < 0 || p >= M_new) {
            atomicOr(&chk->status, 1ull << 2);
            continue;
        }
        e.slot -= E0;
        E_new[p] = e;
        enode_new[p] = v;
    }
}

// New entries go after the kept ones of their node, in slot order.
__global__ void k_scatter_batch(const uint32_t *__restrict__ K, const uint32_t *__restrict__ V, int64_t n,
                                const int32_t *__restrict__ bstart, const int32_t *__restrict__ bcnt,
                                const int32_t *__restrict__ noff_new, const int32_t *__restrict__ src,
                                const int32_t *__restrict__ dst, const int64_t *__restrict__ ts, int directed,
                                int64_t N, int64_t M_new, Entry *E_new, int32_t *enode_new, IngestScratch *chk)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = K[j];
        const uint32_t slot = V[j];
        if ((int64_t)v >= N) {
            atomicOr(&chk->status, 1ull << 3);
            continue;
        }
        const int64_t p = (int64_t)noff_new[v + 1] - bcnt[v] + (j - bstart[v]);
        if (p < 0 || p >= M_new) {
            atomicOr(&chk->status, 1ull << 4);
            continue;
        }
        const int64_t pos = directed ? (int64_t)slot : (int64_t)(slot >> 1);
        const bool side = !directed && (slot & 1u);
        Entry e;
        e.ts = ts[pos];
        e.other = side ? src[pos] : dst[pos];
        e.slot = (int32_t)slot;
        E_new[p] = e;
        enode_new[p] = (int32_t)v;
    }
}

static unsigned grid_for(tempest_t *h, int64_t n, int threads = 256)
{
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)h->num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

void launch_node_off(tempest_t *h, int32_t *node_off)
{
    cudaMemcpyAsync(node_off, h->noff[h->vcur].p, sizeof(int32_t) * (size_t)(h->N + 1), cudaMemcpyDeviceToDevice,
                    h->stream);
}

void launch_node_order(tempest_t *h, int32_t *node_order)
{
    if (h->M > 0)
        k_node_order<<<grid_for(h, h->M), 256, 0, h->stream>>>(h->ent[h->vcur].as<Entry>(), h->M, node_order);
}

static int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

// timestamp-grouped view over the store in buffer h->cur
static int rebuild_ts_view(tempest_t *h)
{
    cudaStream_t st = h->stream;
    const int64_t m = h->m;
    const int64_t *ts = h->st_ts[h->cur].as<int64_t>();
    uint64_t *hpart = static_cast<uint64_t *>(h->hstat);
    int rc;
    if ((rc = ensure(h, h->ts_goff, sizeof(int32_t) * (size_t)(m + 1), true))) return rc;
    TsGroupOp op{ts, h->ts_goff.as<int32_t>()};
    const int nb = scan_launch(op, m, h->partials.as<uint64_t>(), st);
    cudaMemcpyAsync(hpart, h->partials.as<uint64_t>() + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    h->pending_launches += 3;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "ts view"))) return rc;
    h->G = (int64_t)hpart[0];
    k_set_i32<<<1, 1, 0, st>>>(h->ts_goff.as<int32_t>() + h->G, (int32_t)m);
    h->pending_launches++;
    return TEMPEST_OK;
}

static int ensure_view_buffers(tempest_t *h, int nxt, int64_t M, int64_t N)
{
    int rc;
    const size_t Mz = (size_t)(M > 0 ? M : 1);
    if ((rc = ensure(h, h->ent[nxt], sizeof(Entry) * Mz, true))) return rc;
    if ((rc = ensure(h, h->enode[nxt], sizeof(int32_t) * Mz, true))) return rc;
    if ((rc = ensure(h, h->noff[nxt], sizeof(int32_t) * (size_t)(N + 1), true))) return rc;
    if ((rc = ensure(h, h->ngo, sizeof(int32_t) * (size_t)(M + 1), true))) return rc;
    if ((rc = ensure(h, h->ngts, sizeof(int64_t) * Mz, true))) return rc;
    if ((rc = ensure(h, h->gidx, sizeof(int32_t) * (size_t)(N + 1), true))) return rc;
    if ((rc = ensure(h, h->gcnt, sizeof(int32_t) * (size_t)(N + 1), true))) return rc;
    if ((rc = ensure(h, h->seg_node, sizeof(int32_t) * Mz, true))) return rc;
    if ((rc = ensure(h, h->seg_g, sizeof(int32_t) * Mz, true))) return rc;
    return TEMPEST_OK;
}

static int ensure_sort_buffers(tempest_t *h, int64_t n)
{
    int rc;
    const size_t z = (size_t)(n > 0 ? n : 1);
    for (int b = 0; b < 2; b++) {
        if ((rc = ensure(h, h->sk32[b], sizeof(uint32_t) * z, true))) return rc;
        if ((rc = ensure(h, h->sv[b], sizeof(uint32_t) * z, true))) return rc;
    }
    return TEMPEST_OK;
}

// Groups and per-node first groups over the entries in buffer nxt (common to
// both paths); the full path also derives the segment starts from them.
static int node_view_groups(tempest_t *h, int nxt, int64_t M, int64_t N, bool need_noff)
{
    cudaStream_t st = h->stream;
    uint64_t *hpart = static_cast<uint64_t *>(h->hstat);
    int rc;
    {
        NodeGroupOp op{h->enode[nxt].as<int32_t>(), h->ent[nxt].as<Entry>(), h->ngo.as<int32_t>(),
                       h->ngts.as<int64_t>(), h->seg_node.as<int32_t>(), h->seg_g.as<int32_t>()};
        const int nb = scan_launch(op, M, h->partials.as<uint64_t>(), st);
        cudaMemcpyAsync(hpart, h->partials.as<uint64_t>() + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
        h->pending_launches += 3;
    }
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "node view"))) return rc;
    const uint64_t tot = hpart[0];
    const int64_t Gn = M > 0 ? (int64_t)(uint32_t)tot : 0;
    const int64_t S = M > 0 ? (int64_t)(tot >> 32) : 0;
    h->Gn = Gn;
    h->S = S;
    k_set_i32<<<1, 1, 0, st>>>(h->ngo.as<int32_t>() + Gn, (int32_t)M);
    cudaMemsetAsync(h->gcnt.as<int32_t>(), 0, sizeof(int32_t) * (size_t)(N + 1), st);
    if (S > 0)
        k_seg_counts<<<grid_for(h, S), 256, 0, st>>>(h->seg_node.as<int32_t>(), h->seg_g.as<int32_t>(), S, Gn,
                                                     h->gcnt.as<int32_t>());
    {
        GidxOp op{h->gcnt.as<int32_t>(), N, h->gidx.as<int32_t>()};
        scan_launch(op, N + 1, h->partials.as<uint64_t>(), st);
    }
    h->pending_launches += 5;
    if (need_noff) {
        k_node_off<<<grid_for(h, N + 1), 256, 0, st>>>(h->gidx.as<int32_t>(), h->ngo.as<int32_t>(), N,
                                                      h->noff[nxt].as<int32_t>());
        h->pending_launches++;
    }
    return cuda_check(h, cudaGetLastError(), "node view groups");
}

// Full rebuild: stable radix sort of every (node, slot) pair by node.
static int node_view_full(tempest_t *h)
{
    cudaStream_t st = h->stream;
    const int64_t m = h->m;
    const int32_t *src = h->st_src[h->cur].as<int32_t>();
    const int32_t *dst = h->st_dst[h->cur].as<int32_t>();
    const int64_t *ts = h->st_ts[h->cur].as<int64_t>();
    const int64_t M = h->directed ? m : 2 * m;
    const int64_t N = h->N;
    const int nxt = h->vcur ^ 1;
    int rc;
    if ((rc = ensure_view_buffers(h, nxt, M, N))) return rc;
    if ((rc = ensure_sort_buffers(h, M))) return rc;
    if (M > 0) {
        StoreKeyLoader ld{src, dst, h->directed};
        uint32_t *kb[2] = {h->sk32[0].as<uint32_t>(), h->sk32[1].as<uint32_t>()};
        uint32_t *vb[2] = {h->sv[0].as<uint32_t>(), h->sv[1].as<uint32_t>()};
        int launches = 0;
        int bits = bits_for((uint64_t)(N > 0 ? N - 1 : 0));
        if (bits < 1) bits = 1;  // one pass keeps the order and materialises the pairs
        const int r = radix_sort_launch<uint32_t>(ld, M, bits, kb, vb, h->hist.as<uint32_t>(), st, &launches);
        h->pending_launches += launches + 1;
        k_node_entries<<<grid_for(h, M), 256, 0, st>>>(kb[r], vb[r], src, dst, ts, h->directed, M,
                                                       h->ent[nxt].as<Entry>(), h->enode[nxt].as<int32_t>());
    }
    if ((rc = node_view_groups(h, nxt, M, N, true))) return rc;
    h->M = M;
    h->vcur = nxt;
    return TEMPEST_OK;
}

// Incremental update after an append: every node keeps a suffix of its old
// segment (the evicted edges are the oldest) and gains the batch's entries
// at the end.  Gives exactly the order of the full rebuild.
//   i0:   evicted prefix of the old store (in the buffer before h->cur)
//   na:   kept old edges (they are positions [0, na) of the new store)
//   nbk:  batch edges appended at positions [na, na + nbk)
static int node_view_append(tempest_t *h, int64_t i0, int64_t na, int64_t nbk, int64_t N_old, int64_t M_old)
{
    cudaStream_t st = h->stream;
    const int old_store = h->cur ^ 1;
    const int32_t *src = h->st_src[h->cur].as<int32_t>();
    const int32_t *dst = h->st_dst[h->cur].as<int32_t>();
    const int64_t *ts = h->st_ts[h->cur].as<int64_t>();
    const int directed = h->directed;
    const int64_t M = directed ? h->m : 2 * h->m;
    const int64_t N = h->N;
    const int vold = h->vcur, nxt = h->vcur ^ 1;
    const int64_t nbe = directed ? nbk : 2 * nbk;   // new entries
    const int64_t evi = directed ? i0 : 2 * i0;     // evicted entries
    int rc;
    if ((rc = ensure_view_buffers(h, nxt, M, N))) return rc;
    if ((rc = ensure_sort_buffers(h, nbe))) return rc;
    if ((rc = ensure(h, h->ev, sizeof(int32_t) * (size_t)(N + 1), true))) return rc;
    if ((rc = ensure(h, h->bcnt, sizeof(int32_t) * (size_t)(N + 1), true))) return rc;
    if ((rc = ensure(h, h->bstart, sizeof(int32_t) * (size_t)(N + 1), true))) return rc;
    int32_t *ev = h->ev.as<int32_t>();
    int32_t *bcnt = h->bcnt.as<int32_t>();
    int32_t *bstart = h->bstart.as<int32_t>();

    cudaMemsetAsync(ev, 0, sizeof(int32_t) * (size_t)N, st);
    cudaMemsetAsync(bcnt, 0, sizeof(int32_t) * (size_t)N, st);
    if (evi > 0)
        k_evict_counts<<<grid_for(h, evi), 256, 0, st>>>(h->st_src[old_store].as<int32_t>(),
                                                        h->st_dst[old_store].as<int32_t>(), evi, directed, N, ev,
                                                        h->dstat.as<IngestScratch>());
    const uint32_t *Kb = nullptr, *Vb = nullptr;
    if (nbe > 0) {
        BatchKeyLoader ld{src, dst, directed, na};
        uint32_t *kb[2] = {h->sk32[0].as<uint32_t>(), h->sk32[1].as<uint32_t>()};
        uint32_t *vb[2] = {h->sv[0].as<uint32_t>(), h->sv[1].as<uint32_t>()};
        int launches = 0;
        int bits = bits_for((uint64_t)(N > 0 ? N - 1 : 0));
        if (bits < 1) bits = 1;
        const int r = radix_sort_launch<uint32_t>(ld, nbe, bits, kb, vb, h->hist.as<uint32_t>(), st, &launches);
        h->pending_launches += launches;
        Kb = kb[r];
        Vb = vb[r];
        k_batch_runs<<<grid_for(h, nbe), 256, 0, st>>>(Kb, nbe, 0, bstart, bcnt);
        k_batch_runs<<<grid_for(h, nbe), 256, 0, st>>>(Kb, nbe, 1, bstart, bcnt);
        h->pending_launches += 2;
    }
    {
        NoffOp op{h->noff[vold].as<int32_t>(), N_old, ev, bcnt, N, h->noff[nxt].as<int32_t>()};
        scan_launch(op, N + 1, h->partials.as<uint64_t>(), st);
        h->pending_launches += 3;
    }
    if (M_old > 0) {
        k_copy_kept<<<grid_for(h, M_old), 256, 0, st>>>(h->ent[vold].as<Entry>(), h->enode[vold].as<int32_t>(),
                                                       M_old, h->noff[vold].as<int32_t>(), ev,
                                                       h->noff[nxt].as<int32_t>(), (int32_t)evi, N_old, M,
                                                       h->ent[nxt].as<Entry>(), h->enode[nxt].as<int32_t>(),
                                                       h->dstat.as<IngestScratch>());
        h->pending_launches++;
    }
    if (nbe > 0) {
        k_scatter_batch<<<grid_for(h, nbe), 256, 0, st>>>(Kb, Vb, nbe, bstart, bcnt, h->noff[nxt].as<int32_t>(), src,
                                                         dst, ts, directed, N, M, h->ent[nxt].as<Entry>(),
                                                         h->enode[nxt].as<int32_t>(), h->dstat.as<IngestScratch>());
        h->pending_launches++;
    }
    h->pending_launches += (evi > 0) ? 1 : 0;
    if ((rc = node_view_groups(h, nxt, M, N, false))) return rc;
    h->M = M;
    h->vcur = nxt;
    return TEMPEST_OK;
}

int ingest_batch(tempest_t *h, const int32_t *src_in, const int32_t *dst_in, const int64_t *ts_in, int64_t n,
                 tempest_ingest_stats *stats)
{
    cudaStream_t st = h->stream;
    int rc;
    if (n < 0) return fail(h, TEMPEST_EINVAL, "tempest_ingest: n = %lld < 0", (long long)n);
    if (n > 0 && (!src_in || !dst_in || !ts_in)) return fail(h, TEMPEST_EINVAL, "tempest_ingest: NULL array");
    if (n >= (int64_t)INT32_MAX) return fail(h, TEMPEST_EINVAL, "tempest_ingest: batch of %lld edges too large",
                                             (long long)n);
    h->pending_launches = 0;
    h->state_ver++;  // derived walk indexes are rebuilt on the next walk call
    if ((rc = ensure(h, h->dstat, sizeof(IngestScratch)))) return rc;
    if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
    if ((rc = ensure(h, h->hist, sizeof(uint32_t) * ((size_t)RADIX * SORT_MAX_BLOCKS + 1)))) return rc;
    IngestScratch *ds = h->dstat.as<IngestScratch>();
    IngestScratch *hs = static_cast<IngestScratch *>(h->hstat);

    // stage host inputs
    const int32_t *src = src_in;
    const int32_t *dst = dst_in;
    const int64_t *ts = ts_in;
    if (n > 0) {
        if (!is_device_ptr(src_in)) {
            if ((rc = ensure(h, h->b_src, sizeof(int32_t) * (size_t)n, true))) return rc;
            cudaMemcpyAsync(h->b_src.p, src_in, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st);
            src = h->b_src.as<int32_t>();
        }
        if (!is_device_ptr(dst_in)) {
            if ((rc = ensure(h, h->b_dst, sizeof(int32_t) * (size_t)n, true))) return rc;
            cudaMemcpyAsync(h->b_dst.p, dst_in, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st);
            dst = h->b_dst.as<int32_t>();
        }
        if (!is_device_ptr(ts_in)) {
            if ((rc = ensure(h, h->b_ts, sizeof(int64_t) * (size_t)n, true))) return rc;
            cudaMemcpyAsync(h->b_ts.p, ts_in, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, st);
            ts = h->b_ts.as<int64_t>();
        }
    }

    // 1. batch statistics
    k_init_scratch<<<1, 1, 0, st>>>(ds);
    if (n > 0)
        k_batch_stats<<<grid_for(h, n), 256, 0, st>>>(src, dst, ts, n, h->has_cutoff, h->cutoff, ds);
    cudaMemcpyAsync(hs, ds, sizeof(IngestScratch), cudaMemcpyDeviceToHost, st);
    h->pending_launches += 2;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "batch stats"))) return rc;
    if (hs->neg_id) return fail(h, TEMPEST_EINVAL, "tempest_ingest: negative node id");
    const int64_t N_new = (n > 0 && (int64_t)hs->max_id + 1 > h->N) ? (int64_t)hs->max_id + 1 : h->N;
    const int64_t late = (int64_t)hs->late;
    const bool sorted = hs->unsorted == 0;
    const long long bmin = hs->ts_min;
    const uint64_t span = (n > 0) ? (uint64_t)hs->ts_max - (uint64_t)hs->ts_min : 0;

    // capacity of the next state (checked before anything changes)
    const int64_t m_max = h->m + (n - late);
    const int64_t M_max = h->directed ? m_max : 2 * m_max;
    if (M_max >= (int64_t)INT32_MAX - 1)
        return fail(h, TEMPEST_ENOMEM, "tempest_ingest: %lld index entries exceed the int32 index range",
                    (long long)M_max);

    // 2. sort the batch by timestamp (stable), late edges become a prefix
    const int32_t *bs = src;
    const int32_t *bd = dst;
    const int64_t *bt = ts;
    if (n > 0 && !sorted) {
        if ((rc = ensure(h, h->sk64[0], sizeof(uint64_t) * (size_t)n, true))) return rc;
        if ((rc = ensure(h, h->sk64[1], sizeof(uint64_t) * (size_t)n, true))) return rc;
        if ((rc = ensure(h, h->sv[0], sizeof(uint32_t) * (size_t)n, true))) return rc;
        if ((rc = ensure(h, h->sv[1], sizeof(uint32_t) * (size_t)n, true))) return rc;
        if ((rc = ensure(h, h->sb_src, sizeof(int32_t) * (size_t)n, true))) return rc;
        if ((rc = ensure(h, h->sb_dst, sizeof(int32_t) * (size_t)n, true))) return rc;
        if ((rc = ensure(h, h->sb_ts, sizeof(int64_t) * (size_t)n, true))) return rc;
        TsKeyLoader ld{ts, bmin};
        unsigned long long *kb[2] = {h->sk64[0].as<unsigned long long>(), h->sk64[1].as<unsigned long long>()};
        uint32_t *vb[2] = {h->sv[0].as<uint32_t>(), h->sv[1].as<uint32_t>()};
        int launches = 0;
        const int r = radix_sort_launch<unsigned long long>(ld, n, bits_for(span), kb, vb, h->hist.as<uint32_t>(),
                                                            st, &launches);
        h->pending_launches += launches;
        // span > 0 whenever the batch is unsorted, so a pass ran
        k_gather_batch<<<grid_for(h, n), 256, 0, st>>>(vb[r], src, dst, ts, n, h->sb_src.as<int32_t>(),
                                                       h->sb_dst.as<int32_t>(), h->sb_ts.as<int64_t>());
        h->pending_launches++;
        bs = h->sb_src.as<int32_t>();
        bd = h->sb_dst.as<int32_t>();
        bt = h->sb_ts.as<int64_t>();
    }
    bs += late;
    bd += late;
    bt += late;
    const int64_t nb = n - late;

    // 3. window cut-off
    const int mode = h->window > 0 ? 1 : (h->window < 0 ? 2 : 0);
    const long long param = h->window > 0 ? h->window : -h->window;
    const int64_t *old_ts = h->st_ts[h->cur].as<int64_t>();
    k_window<<<1, 32, 0, st>>>(mode, param, old_ts, h->m, bt, nb, h->has_cutoff, h->cutoff, ds);
    cudaMemcpyAsync(hs, ds, sizeof(IngestScratch), cudaMemcpyDeviceToHost, st);
    h->pending_launches++;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "window"))) return rc;
    const int64_t i0 = hs->i0, j0 = hs->j0;
    const int64_t na = h->m - i0, nbk = nb - j0;
    const int64_t m_new = na + nbk;

    // 4. merge into the other store buffer
    const int nxt = h->cur ^ 1;
    const bool append = na == 0 || nbk == 0 || hs->store_last_ts <= hs->kept_batch_min_ts;
    if ((rc = ensure(h, h->st_src[nxt], sizeof(int32_t) * (size_t)(m_new > 0 ? m_new : 1), true))) return rc;
    if ((rc = ensure(h, h->st_dst[nxt], sizeof(int32_t) * (size_t)(m_new > 0 ? m_new : 1), true))) return rc;
    if ((rc = ensure(h, h->st_ts[nxt], sizeof(int64_t) * (size_t)(m_new > 0 ? m_new : 1), true))) return rc;
    {
        const int32_t *as = h->st_src[h->cur].as<int32_t>() + i0;
        const int32_t *ad = h->st_dst[h->cur].as<int32_t>() + i0;
        const int64_t *at = h->st_ts[h->cur].as<int64_t>() + i0;
        int32_t *os = h->st_src[nxt].as<int32_t>();
        int32_t *od = h->st_dst[nxt].as<int32_t>();
        int64_t *ot = h->st_ts[nxt].as<int64_t>();
        if (append) {
            if (na > 0) {
                cudaMemcpyAsync(os, as, sizeof(int32_t) * (size_t)na, cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(od, ad, sizeof(int32_t) * (size_t)na, cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(ot, at, sizeof(int64_t) * (size_t)na, cudaMemcpyDeviceToDevice, st);
            }
            if (nbk > 0) {
                cudaMemcpyAsync(os + na, bs + j0, sizeof(int32_t) * (size_t)nbk, cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(od + na, bd + j0, sizeof(int32_t) * (size_t)nbk, cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(ot + na, bt + j0, sizeof(int64_t) * (size_t)nbk, cudaMemcpyDeviceToDevice, st);
            }
        } else {
            const int64_t threads = (m_new + MERGE_K - 1) / MERGE_K;
            k_merge<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(as, ad, at, na, bs + j0, bd + j0, bt + j0, nbk,
                                                                       os, od, ot);
            h->pending_launches++;
        }
    }
    if ((rc = cuda_check(h, cudaGetLastError(), "merge"))) return rc;

    // commit the new store and counters
    const int64_t N_old = h->N, M_old = h->M;
    h->cur = nxt;
    h->m = m_new;
    h->N = N_new;
    h->seq_next += n;
    h->dropped += late;
    h->evicted += i0 + j0;
    const int64_t evicted_now = i0 + j0;
    h->has_cutoff = hs->has_cut;
    h->cutoff = hs->cut;

    // 5-6. views: incremental node view after an append, full rebuild after
    // a general merge (or before any view exists)
    if ((rc = rebuild_ts_view(h))) return rc;
    if (append && h->ent[h->vcur].p) rc = node_view_append(h, i0, na, nbk, N_old, M_old);
    else rc = node_view_full(h);
    if (rc) return rc;
    cudaMemcpyAsync(hs, ds, sizeof(IngestScratch), cudaMemcpyDeviceToHost, st);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "ingest"))) return rc;
    if (hs->status)
        return fail(h, TEMPEST_ECUDA, "ingest: index consistency check failed (code 0x%llx)",
                    (unsigned long long)hs->status);

    if (stats) {
        stats->n_in = n;
        stats->n_dropped_late = late;
        stats->n_evicted = evicted_now;
        stats->n_live = h->m;
        stats->n_ts_groups = h->G;
        stats->n_node_groups = h->Gn;
        stats->n_nodes = h->N;
        stats->cutoff = h->cutoff;
        stats->has_cutoff = h->has_cutoff;
        stats->sorted_input = sorted ? 1 : 0;
        stats->launches = h->pending_launches;
    }
    return TEMPEST_OK;
}

}  // namespace tw
