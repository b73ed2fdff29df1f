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
//   4. when the kept batch starts no earlier than the store ends (a stream in
//      time order), eviction only advances the store's head and the batch is
//      appended at its tail; the live range moves to the front of the other
//      buffer only when the tail reaches the end (amortised: the buffer holds
//      twice the live edges).  Otherwise the kept store and batch are merged
//      into the other buffer (merge-path merge);
//   5. timestamp-grouped view: eviction advances its first live group (a
//      binary search), the batch's group starts are appended (a compaction
//      over the batch only); after a merge or a move it is rebuilt;
//   6. node view (nodeview.cu): per-node regions updated by the batch and the
//      evicted edges only, or rebuilt from the store after a merge.
#include <stdio.h>

#include <algorithm>

#include "engine.cuh"
#include "prims.cuh"
#include "sortscan.cuh"

namespace tw {

// ---------------------------------------------------------------------------
// batch statistics
// ---------------------------------------------------------------------------
// One pass over the batch: timestamp range, largest id, reserved values,
// late edges, whether the timestamps already ascend, and a byte per edge
// that says whether its timestamp differs from the edge before it (for a
// batch that arrives sorted, the starts of its timestamp groups).  Each thread keeps
// four loads of each array in flight (grid-stride, unrolled); each warp and
// then each block reduce in registers and shared memory, so the global
// atomics are one set per block (per-warp atomics on the same six words
// serialised at L2).  With os / od / ot set (the store's free tail, when it
// has room for the whole batch) it also writes the batch there: a batch that
// proves sorted, on time and wholly kept is then appended without a second
// read (the store copies were 320 MB of traffic per 10M edges); otherwise
// the append overwrites that free space.
constexpr int STATS_THREADS = 256;
constexpr int STATS_UNROLL = 4;

__global__ void __launch_bounds__(STATS_THREADS) k_batch_stats(const int32_t *__restrict__ src,
                                                               const int32_t *__restrict__ dst,
                                                               const int64_t *__restrict__ ts, int64_t n,
                                                               int has_cut, long long cut, uint8_t *gflag,
                                                               int32_t *os, int32_t *od, int64_t *ot,
                                                               IngestScratch *o)
{
    long long tmin = LLONG_MAX, tmax = LLONG_MIN;
    int maxid = 0, neg = 0;
    unsigned long long late = 0, uns = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * STATS_UNROLL) {
        int32_t a[STATS_UNROLL], b[STATS_UNROLL];
        long long t[STATS_UNROLL], tp[STATS_UNROLL];
#pragma unroll
        for (int r = 0; r < STATS_UNROLL; r++) {
            const int64_t i = i0 + r * stride;
            const bool ok = i < n;
            a[r] = ok ? __ldg(src + i) : 0;
            b[r] = ok ? __ldg(dst + i) : 0;
            t[r] = ok ? __ldg(ts + i) : 0;
            tp[r] = (ok && i > 0) ? __ldg(ts + i - 1) : LLONG_MIN;
        }
#pragma unroll
        for (int r = 0; r < STATS_UNROLL; r++) {
            if (i0 + r * stride >= n) continue;
            tmin = min(tmin, t[r]);
            tmax = max(tmax, t[r]);
            maxid = max(maxid, max(a[r], b[r]));
            neg |= (a[r] < 0) | (b[r] < 0) | ((t[r] == LLONG_MIN) ? 2 : 0) | ((t[r] == LLONG_MAX) ? 4 : 0);
            late += (has_cut && t[r] < cut) ? 1ull : 0ull;
            uns += tp[r] > t[r] ? 1ull : 0ull;
            // a timestamp group starts here (against the batch's previous
            // edge; the first kept edge is compared with the store later)
            gflag[i0 + r * stride] = tp[r] != t[r] ? 1 : 0;
            if (os) {  // the store's tail, in case the batch is appended as it is
                os[i0 + r * stride] = a[r];
                od[i0 + r * stride] = b[r];
                ot[i0 + r * stride] = t[r];
            }
        }
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
    constexpr int W = STATS_THREADS / 32;
    __shared__ long long s_min[W], s_max[W];
    __shared__ int s_id[W], s_neg[W];
    __shared__ unsigned long long s_late[W], s_uns[W];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_min[w] = tmin;
        s_max[w] = tmax;
        s_id[w] = maxid;
        s_neg[w] = neg;
        s_late[w] = late;
        s_uns[w] = uns;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < W; k++) {
            tmin = min(tmin, s_min[k]);
            tmax = max(tmax, s_max[k]);
            maxid = max(maxid, s_id[k]);
            neg |= s_neg[k];
            late += s_late[k];
            uns += s_uns[k];
        }
        atomicMin(&o->ts_min, tmin);
        atomicMax(&o->ts_max, tmax);
        atomicMax(&o->max_id, maxid);
        if (neg) atomicOr(&o->neg_id, neg);
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
    o->tg_lo = 0;
    o->tg_added = 0;
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
// First index in [lo, hi) where a monotone predicate (false ... false true
// ... true) holds, hi if none, found by the 32 lanes of a warp together: each
// step probes 32 evenly spaced points of the bracket, so a search over 2^28
// elements takes 6 dependent loads instead of 28.  Every lane returns the
// answer.
template <class Pred>
__device__ __forceinline__ int64_t warp_partition_point(int64_t lo, int64_t hi, const Pred &pred)
{
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const int64_t w = hi - lo;
        const int64_t pnt = lo + (w * (lane + 1)) / 33;  // strictly inside [lo, hi)
        const unsigned t = __ballot_sync(0xffffffffu, pred(pnt));
        const int c = __popc(~t);  // probes where the predicate is false: a prefix
        const int64_t plo = c > 0 ? lo + (w * c) / 33 + 1 : lo;        // after the last false probe
        const int64_t phi = c < 32 ? lo + (w * (c + 1)) / 33 : hi;     // the first true probe
        lo = plo;
        hi = phi;
    }
    const int64_t q = lo + lane;
    const unsigned t = __ballot_sync(0xffffffffu, q < hi && !pred(q));
    return lo + __popc(t);
}

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
// With `fused` the kernel runs right after k_batch_stats on the batch as it
// came: when the statistics found it sorted, its late edges are the first
// o->late ones and the window is computed on the rest (one host round trip
// for both steps); an unsorted batch is left to a second launch on the
// sorted batch.
__global__ void k_window(int mode, long long param, const int64_t *old_ts, int64_t m_old,
                         const int64_t *bts, int64_t nb, int has_old, long long cut_old, int fused, IngestScratch *o)
{
    // one warp: lane 0's results are written; the searches run on all lanes
    if (threadIdx.x >= 32 || blockIdx.x != 0) return;
    if (fused) {
        if (o->unsorted) return;
        const int64_t late = (int64_t)o->late;
        bts += late;
        nb -= late;
    }
    int has = has_old;
    long long cut = cut_old;
    const int lane = threadIdx.x;
    if (mode == 1 && m_old + nb > 0) {
        long long tmax = LLONG_MIN;
        if (m_old > 0) tmax = old_ts[m_old - 1];
        if (nb > 0) tmax = max(tmax, (long long)bts[nb - 1]);
        const long long c = (tmax < LLONG_MIN + param) ? LLONG_MIN : tmax - param;
        if (!has || c > cut) cut = c;
        has = 1;
    } else if (mode == 2 && m_old + nb > param) {
        const int64_t r = m_old + nb - param;  // rank of the W-th newest element
        // merge split: the first i with a[i] after b[r - i - 1] (see merge_split)
        const int64_t i = warp_partition_point(r > nb ? r - nb : 0, r < m_old ? r : m_old, [&](int64_t x) {
            const int64_t jj = r - x;
            return jj == 0 || bts[jj - 1] < old_ts[x];
        });
        const int64_t j = r - i;
        long long c;
        if (j >= nb || (i < m_old && old_ts[i] <= bts[j])) c = old_ts[i];
        else c = bts[j];
        if (!has || c > cut) cut = c;
        has = 1;
    }
    int64_t i0 = 0, j0 = 0;
    if (has) {
        i0 = warp_partition_point(0, m_old, [&](int64_t x) { return old_ts[x] >= cut; });
        j0 = warp_partition_point(0, nb, [&](int64_t x) { return bts[x] >= cut; });
    }
    if (lane != 0) return;
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
// timestamp-grouped view
// ---------------------------------------------------------------------------
// Group starts among the store indices [lo, lo + n) of ts: a group opens
// where the timestamp differs from the previous edge's, and at index first
// (the live head).  Starts are written densely from tg as absolute store
// positions modulo 2^32 (abs0 is the absolute position of index 0), so a
// move of the store's live range does not change them.
struct TsGroupOp {
    const int64_t *ts;
    int64_t lo, first;
    uint32_t abs0;
    int32_t *tg;
    __device__ __forceinline__ uint64_t value(int64_t i) const
    {
        const int64_t p = lo + i;
        return (p == first || ts[p] != ts[p - 1]) ? 1u : 0u;
    }
    __device__ __forceinline__ void emit(int64_t i, uint64_t v, uint64_t ex) const
    {
        if (v) tg[ex] = (int32_t)(abs0 + (uint32_t)(lo + i));
    }
};

// The same starts for a batch that arrived sorted, from the batch statistics'
// bytes: the flag of kept edge i (i >= 1) is base[a + i] (base 16-byte
// aligned); the first kept edge is compared with the store's previous edge.
// A byte scan (16 flags per thread, one load) instead of two timestamps per
// edge on both scan passes.
struct TsTailBytes {
    const uint8_t *base;
    int64_t a, n;
    const int64_t *ts;
    int64_t lo, first;
    uint32_t abs0;
    int32_t *tg;
    struct Stage {
        int32_t v[BSCAN_TILE];  // the tile's group starts, written out coalesced
    };
    __host__ __device__ int64_t tiles() const { return n > 0 ? (a + n + BSCAN_TILE - 1) / BSCAN_TILE : 0; }
    __device__ __forceinline__ uint4 load(int64_t u0) const
    {
        return u0 < a + n ? __ldg(reinterpret_cast<const uint4 *>(base + u0)) : make_uint4(0, 0, 0, 0);
    }
    __device__ __forceinline__ uint32_t mask16(uint4 w, int64_t u0) const
    {
        uint32_t m = byte_bits16(w, 0) & valid16(u0, a, n);
        if (u0 <= a && a < u0 + 16) {  // the first kept edge against the store's edge before it
            const int k = (int)(a - u0);
            const bool f = lo == first || ts[lo] != ts[lo - 1];
            m = (m & ~(1u << k)) | ((f ? 1u : 0u) << k);
        }
        return m;
    }
    __device__ __forceinline__ uint64_t sum16(uint4 w, int64_t u0) const { return (uint64_t)__popc(mask16(w, u0)); }
    __device__ __forceinline__ void emit16(uint4 w, int64_t u0, uint64_t ex, uint64_t tile_ex, uint64_t tile_tot,
                                           Stage &sm) const
    {
        uint32_t m = mask16(w, u0);
        int j = (int)(ex - tile_ex);
        const uint32_t v0 = abs0 + (uint32_t)(lo + (u0 - a));
        while (m) {
            const int k = __ffs(m) - 1;
            m &= m - 1;
            sm.v[j++] = (int32_t)(v0 + (uint32_t)k);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < (int)tile_tot; q += blockDim.x) tg[tile_ex + q] = sm.v[q];
        __syncthreads();
    }
};

// First live group after the head moved to absolute position s_lo: the first
// g in [lo, hi) whose successor starts after s_lo (tg[hi] is the old tail),
// else hi.  Positions compare modulo 2^32 (the live span is below 2^31).
__global__ void k_ts_evict(const int32_t *__restrict__ tg, int64_t lo, int64_t hi, uint32_t s_lo, IngestScratch *o)
{
    if (threadIdx.x >= 32) return;  // one warp
    const int64_t g = warp_partition_point(lo, hi, [&](int64_t x) { return (int32_t)((uint32_t)tg[x + 1] - s_lo) > 0; });
    if (threadIdx.x == 0) o->tg_lo = g;
}

// After a compaction of n appended starts written from tg + base: the tail
// entry (absolute end of the store) and the count.
__global__ void k_ts_tail(int32_t *tg, int64_t base, const uint64_t *tot, uint32_t s_hi, IngestScratch *o)
{
    const uint64_t n = *tot;
    tg[base + (int64_t)n] = (int32_t)s_hi;
    o->tg_added = (long long)n;
}

static unsigned grid_for(tempest_t *h, int64_t n, int threads = 256)
{
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)h->num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

static int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

static uint32_t abs32(const tempest_t *h, int64_t idx) { return (uint32_t)(uint64_t)(h->s_base + idx); }

// Timestamp view over the whole live range of buffer cur.
static int ts_view_build(tempest_t *h)
{
    cudaStream_t st = h->stream;
    const int64_t m = h->s_hi - h->s_lo;
    int rc;
    if ((rc = ensure(h, h->tg, sizeof(int32_t) * (size_t)(2 * m + 1024), true))) return rc;
    IngestScratch *ds = h->dstat.as<IngestScratch>();
    TsGroupOp op{h->st_ts[h->cur].as<int64_t>(), h->s_lo, h->s_lo, abs32(h, 0), h->tg.as<int32_t>()};
    const int nb = scan_launch(op, m, h->partials.as<uint64_t>(), st);
    k_ts_tail<<<1, 1, 0, st>>>(h->tg.as<int32_t>(), 0, h->partials.as<uint64_t>() + nb, abs32(h, h->s_hi), ds);
    h->pending_launches += 4;
    h->tg_lo = 0;
    h->tg_hi = -1;  // known after the batch's final read-back (tg_added)
    return cuda_check(h, cudaGetLastError(), "ts view");
}

__global__ void k_ts_export(const int32_t *__restrict__ tg, int64_t G, uint32_t s_lo, int64_t m, int32_t *out)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += (int64_t)gridDim.x * blockDim.x)
        out[g] = g < G ? max((int32_t)((uint32_t)tg[g] - s_lo), 0) : (int32_t)m;
}

int ts_export(tempest_t *h, int32_t *out)
{
    k_ts_export<<<grid_for(h, h->G + 1), 256, 0, h->stream>>>(h->tg.as<int32_t>() + h->tg_lo, h->G,
                                                              abs32(h, h->s_lo), h->m, out);
    return cuda_check(h, cudaGetLastError(), "export");
}

// Batches before a full store buffer during which each appending batch copies
// a share of the live range to the other buffer (the move then copies only
// the last share: no 3 GB copy in one batch of a 200M-edge window), for live
// ranges of at least the copy-ahead threshold (TEMPEST_TUNE_MIRROR_MIN).
constexpr int64_t STORE_PRECOPY = 6;

// Store capacity a count window settles at (the live edges never exceed the
// window by more than a tie group, so this is the size the store grows to):
// allocating it once the live edges reach 1/16 of the window spares the
// steady state the reallocation of a buffer, which synchronises the device
// and stalls a batch.  Duration windows, unbounded stores and windows far
// above the content grow with their content instead (0).
static int64_t steady_store_cap(const tempest_t *h, int64_t m_new, int64_t nbk)
{
    if (h->window >= 0) return 0;
    const int64_t W = -h->window;
    if (W > 16 * (m_new + nbk)) return 0;
    return 2 * W + W / 2 + nbk + 1024;
}

// Algorithmic bytes of one ingest in this design: each array the batch
// touches, read or written once for its role, per-node records at their
// size (not the sectors a random access occupies).  b = batch edges, k =
// kept edges, E / P / U / R = the node view's appended entries, radix
// passes, distinct nodes and node runs, e / u = evicted entries and the
// nodes that lost them:
//   17 b                 batch statistics (src, dst, ts read; a group-start
//                        byte written per edge)
//   P_ts (24 b) + 32 b   timestamp sort of an unsorted batch (8-byte key and
//                        4-byte index read and written per pass), gather
//   32 k                 store append (kept batch read, store written; 16 k
//                        when the batch statistics wrote the store as they
//                        read the batch); a merge instead reads both sides
//                        and writes the store
//   32 s + 8 t           live edges copied to the other store buffer (a move,
//                        or a share of one copied ahead), live timestamp-view
//                        starts moved to a larger buffer
//   2 k + 4 G_new        timestamp view (both scan passes read the kept
//                        edges' group-start bytes; 16 k when the batch came
//                        unsorted and its timestamps are read instead)
//   4 e + 104 u          eviction: endpoint ids read; per node its counter
//                        (8) and its records (16 + 32) read and written (32 A
//                        + 96 u when the A active nodes search their own
//                        entries instead: record and first entry read per
//                        node, no ids read, no counter)
//   4 E + 16 U           batch-local ids (ids read, id table)
//   20 P E               node sort passes (key read for the histogram, key
//                        and value read and written by the scatter; the
//                        first pass's histogram writes the keys its scatter
//                        reads, and its values are the indices, read by none)
//   41 E                 entries packed in sorted order (index and key
//                        read, the store item's far end and time gathered,
//                        16-byte entry and a run/group-start byte written)
//   2 E + 148 R          runs (both scan passes read the start bytes; per
//                        run its arrays, node record and the region
//                        reservation)
//   32 E_moved + 24 G_moved   region moves (entries, group starts and times)
//   33 E + 12 G_added    scatter (the start byte and the packed entry read,
//                        the entry and new groups written)
// A full rebuild of the node view (after a merge or a pool exhaustion)
// counts its whole sort and scatter over the live entries instead.
static int64_t ingest_model_bytes(const NvBatchReport &r, int64_t b, int64_t k, int64_t kept_old, int64_t m_new,
                                  int ts_passes, bool append, bool store_fused, bool ts_full, int64_t tg_added,
                                  int64_t G, int64_t store_moved, int64_t ts_moved)
{
    int64_t x = 17 * b + 32 * store_moved + 8 * ts_moved;
    if (ts_passes > 0) x += ts_passes * 24 * b + 32 * b;
    x += append ? (store_fused ? 16 * k : 32 * k) : 16 * (kept_old + k) + 16 * m_new;
    x += ts_full ? 16 * m_new + 4 * G : (ts_passes > 0 ? 16 * k : 2 * k) + 4 * tg_added;
    if (r.rebuilt) {
        const int64_t M = r.rb_entries;
        x += M * (8 + 20 * r.rb_passes + 32 + 32 + 32) + 12 * r.rb_groups + 104 * r.rb_nodes;
    } else {
        x += r.ev_scanned ? 32 * r.ev_scanned + 96 * r.ev_nodes : 4 * r.ev_entries + 104 * r.ev_nodes;
        x += 4 * r.entries + 16 * r.ids;
        x += 20 * r.passes * r.entries;
        x += 41 * r.entries;
        x += 2 * r.entries + 148 * r.runs;
        x += 32 * r.moved_e + 24 * r.moved_g;
        x += 33 * r.entries + 12 * r.g_added;
    }
    return x;
}

static IngestUndo undo_record(const tempest_t *h)
{
    IngestUndo u;
    u.m = h->m;
    u.G = h->G;
    u.N = h->N;
    u.M = h->M;
    u.Gn = h->Gn;
    u.dropped = h->dropped;
    u.evicted = h->evicted;
    u.seq_next = h->seq_next;
    u.cutoff = h->cutoff;
    u.s_lo = h->s_lo;
    u.s_hi = h->s_hi;
    u.s_cap = h->s_cap;
    u.s_base = h->s_base;
    u.tg_lo = h->tg_lo;
    u.tg_hi = h->tg_hi;
    u.n_act = h->n_act;
    u.S = h->S;
    u.has_cutoff = h->has_cutoff;
    u.cur = h->cur;
    return u;
}

void ingest_undo(tempest_t *h, const IngestUndo &u)
{
    h->m = u.m;
    h->G = u.G;
    h->N = u.N;
    h->M = u.M;
    h->Gn = u.Gn;
    h->dropped = u.dropped;
    h->evicted = u.evicted;
    h->seq_next = u.seq_next;
    h->cutoff = u.cutoff;
    h->s_lo = u.s_lo;
    h->s_hi = u.s_hi;
    h->s_cap = u.s_cap;
    h->s_base = u.s_base;
    h->tg_lo = u.tg_lo;
    h->tg_hi = u.tg_hi;
    h->n_act = u.n_act;
    h->S = u.S;
    h->has_cutoff = u.has_cutoff;
    h->cur = u.cur;
    h->smir_on = false;  // the other buffer may have been written past the copy's record
    h->tmir_on = false;
    // the views may hold part of the undone batch: rebuilt from the store
    h->nv_ready = false;
    h->w_valid = false;
    h->views_dirty = true;
    h->state_ver++;
}

static int views_rebuild(tempest_t *h);

int views_repair(tempest_t *h)
{
    if (!h->views_dirty) return TEMPEST_OK;
    // the rebuild resets the view counters before it allocates: keep them
    // for a rebuild that fails (the state the counters describe is unchanged)
    const IngestUndo u = undo_record(h);
    const int rc = views_rebuild(h);
    if (rc) {
        ingest_undo(h, u);
        return rc;
    }
    return TEMPEST_OK;
}

static int views_rebuild(tempest_t *h)
{
    cudaStream_t st = h->stream;
    int rc;
    if ((rc = ensure(h, h->dstat, sizeof(IngestScratch)))) return rc;
    if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
    if ((rc = ensure(h, h->hist, sizeof(uint32_t) * (size_t)SORT_HIST_WORDS))) return rc;
    IngestScratch *ds = h->dstat.as<IngestScratch>();
    IngestScratch *hs = static_cast<IngestScratch *>(h->hstat);
    h->state_ver++;
    if (h->m == 0) {
        // the state of a handle with no live edge: empty views, built by the
        // next ingest
        h->tg_lo = h->tg_hi = 0;
        h->G = 0;
        h->views_dirty = false;
        return TEMPEST_OK;
    }
    k_init_scratch<<<1, 1, 0, st>>>(ds);
    if ((rc = ts_view_build(h))) return rc;
    cudaMemcpyAsync(hs, ds, sizeof(IngestScratch), cudaMemcpyDeviceToHost, st);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "view repair"))) return rc;
    h->tg_lo = 0;
    h->tg_hi = hs->tg_added;
    h->G = h->tg_hi;
    if ((rc = nv_build(h))) return rc;
    if (h->pt_on) {
        if ((rc = pt_rebuild(h, &ds->status))) return rc;
        cudaMemcpyAsync(hs, ds, sizeof(IngestScratch), cudaMemcpyDeviceToHost, st);
        if ((rc = cuda_check(h, cudaStreamSynchronize(st), "view repair"))) return rc;
        if (hs->status)
            return fail(h, TEMPEST_ECUDA, "view repair: pair table check failed (code 0x%llx)",
                        (unsigned long long)hs->status);
    }
    h->views_dirty = false;
    return TEMPEST_OK;
}

static int ingest_batch_impl(tempest_t *h, const int32_t *src_in, const int32_t *dst_in, const int64_t *ts_in,
                             int64_t n, tempest_ingest_stats *stats, bool *changing);

int ingest_batch(tempest_t *h, const int32_t *src_in, const int32_t *dst_in, const int64_t *ts_in, int64_t n,
                 tempest_ingest_stats *stats, IngestUndo *undo)
{
    NvtxRange range("tempest_ingest");
    int rc = views_repair(h);
    if (rc) return rc;
    const IngestUndo u = undo_record(h);
    bool changing = false;
    rc = ingest_batch_impl(h, src_in, dst_in, ts_in, n, stats, &changing);
    if (rc == TEMPEST_OK) {
        if (undo) *undo = u;
        return rc;
    }
    // nothing to undo when the call failed before it began to change the state
    if (changing) {
        // keep the first error's message: the repair is best effort here (a
        // repair that fails again is retried by the next call)
        const std::string msg = h->err;
        ingest_undo(h, u);
        views_repair(h);
        h->err = msg;
    }
    return rc;
}

static int ingest_batch_impl(tempest_t *h, const int32_t *src_in, const int32_t *dst_in, const int64_t *ts_in,
                             int64_t n, tempest_ingest_stats *stats, bool *changing)
{
    NvtxStages stage;
    stage.next("ingest: stage inputs");
    h->nv_rep = NvBatchReport{};
    cudaStream_t st = h->stream;
    int rc;
    if (n < 0) return fail(h, TEMPEST_EINVAL, "tempest_ingest: n = %lld < 0", (long long)n);
    if (n > 0 && (!src_in || !dst_in || !ts_in)) return fail(h, TEMPEST_EINVAL, "tempest_ingest: NULL array");
    if (n >= (int64_t)INT32_MAX) return fail(h, TEMPEST_EINVAL, "tempest_ingest: batch of %lld edges too large",
                                             (long long)n);
    h->pending_launches = 0;
    h->eev_valid = false;
    h->state_ver++;  // derived walk indexes are rebuilt on the next walk call
    if ((rc = ensure(h, h->dstat, sizeof(IngestScratch)))) return rc;
    if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
    if ((rc = ensure(h, h->hist, sizeof(uint32_t) * (size_t)SORT_HIST_WORDS))) return rc;
    if ((rc = ensure(h, h->b_gflag, (size_t)n + 1, true))) return rc;
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
    stage.next("ingest: batch statistics");
    k_init_scratch<<<1, 1, 0, st>>>(ds);
    // the store's free tail takes the batch as it is read (used when the
    // batch turns out to be appended whole; nothing reads that space else)
    const bool spec = n > 0 && h->st_src[h->cur].p && h->s_hi + n <= h->s_cap;
    const int64_t spec_at = h->s_hi;
    if (n > 0)
        k_batch_stats<<<std::min<unsigned>(grid_for(h, (n + STATS_UNROLL - 1) / STATS_UNROLL, STATS_THREADS),
                                           (unsigned)h->num_sms * 4),
                        STATS_THREADS, 0, st>>>(
            src, dst, ts, n, h->has_cutoff, h->cutoff, h->b_gflag.as<uint8_t>(),
            spec ? h->st_src[h->cur].as<int32_t>() + spec_at : nullptr,
            spec ? h->st_dst[h->cur].as<int32_t>() + spec_at : nullptr,
            spec ? h->st_ts[h->cur].as<int64_t>() + spec_at : nullptr, ds);
    // the window of a batch that turns out sorted (the usual stream), in the
    // same round trip
    const int mode = h->window > 0 ? 1 : (h->window < 0 ? 2 : 0);
    const long long param = h->window > 0 ? h->window : -h->window;
    const int64_t *old_ts = h->m > 0 ? h->st_ts[h->cur].as<int64_t>() + h->s_lo : nullptr;
    k_window<<<1, 32, 0, st>>>(mode, param, old_ts, h->m, ts, n, h->has_cutoff, h->cutoff, 1, ds);
    cudaMemcpyAsync(hs, ds, sizeof(IngestScratch), cudaMemcpyDeviceToHost, st);
    h->pending_launches += 3;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "batch stats"))) return rc;
    if (hs->neg_id & 1) return fail(h, TEMPEST_EINVAL, "tempest_ingest: negative node id");
    if (hs->neg_id & 2) return fail(h, TEMPEST_EINVAL, "tempest_ingest: timestamp INT64_MIN is reserved");
    if (hs->neg_id & 4) return fail(h, TEMPEST_EINVAL, "tempest_ingest: timestamp INT64_MAX is reserved");
    const int64_t N_new = (n > 0 && (int64_t)hs->max_id + 1 > h->N) ? (int64_t)hs->max_id + 1 : h->N;
    const int64_t late = (int64_t)hs->late;
    const bool sorted = hs->unsorted == 0;
    const long long bmin = hs->ts_min;
    const uint64_t span = (n > 0) ? (uint64_t)hs->ts_max - (uint64_t)hs->ts_min : 0;

    // capacity of the next state (checked before anything changes)
    const int64_t m_max = h->m + (n - late);
    const int64_t M_max = h->directed ? m_max : 2 * m_max;
    if (M_max >= (int64_t)INT32_MAX / 2)
        return fail(h, TEMPEST_ENOMEM, "tempest_ingest: %lld index entries exceed the int32 index range",
                    (long long)M_max);

    // 2. sort the batch by timestamp (stable), late edges become a prefix
    stage.next("ingest: batch sort");
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
    stage.next("ingest: window cut-off");
    if (!sorted) {
        k_window<<<1, 32, 0, st>>>(mode, param, old_ts, h->m, bt, nb, h->has_cutoff, h->cutoff, 0, ds);
        cudaMemcpyAsync(hs, ds, sizeof(IngestScratch), cudaMemcpyDeviceToHost, st);
        h->pending_launches++;
        if ((rc = cuda_check(h, cudaStreamSynchronize(st), "window"))) return rc;
    }
    const int64_t i0 = hs->i0, j0 = hs->j0;
    const int64_t na = h->m - i0, nbk = nb - j0;
    const int64_t m_new = na + nbk;
    const bool append = na == 0 || nbk == 0 || hs->store_last_ts <= hs->kept_batch_min_ts;

    // 4. the allocations of the steps below, made before anything changes:
    // a call whose memory runs short fails here and leaves the state as it
    // was, without a rebuild (only a node view pool that proves too small,
    // and the Node2Vec pair table, allocate later)
    stage.next("ingest: reserve");
    const int64_t N_old = h->N;
    const int old_buf = h->cur;
    const int64_t old_lo = h->s_lo;
    bool ts_full = !append || !h->tg.p || h->views_dirty;
    bool nv_full = !append || !h->nv_ready;
    // an appending batch into a buffer that fills within STORE_PRECOPY
    // batches copies a share of the live range to the other buffer (below)
    const bool store_full = append && h->s_hi + nbk > h->s_cap;
    // the timestamp view's starts move to a larger buffer when the batch's
    // cannot follow them; in the TS_PRECOPY batches before, each copies a
    // share ahead (as the store)
    const int64_t tg_room = (int64_t)(h->tg.bytes / sizeof(int32_t)) - h->tg_hi - 2;
    const bool ts_move = !ts_full && tg_room < nbk;
    const bool ts_precopy = !ts_full && !ts_move && nbk > 0 && h->tg_hi - h->tg_lo >= h->mirror_min &&
                            (h->tmir_on || tg_room < STORE_PRECOPY * nbk);
    const bool precopy = append && !store_full && nbk > 0 && na >= h->mirror_min &&
                         (h->smir_on || h->s_cap - h->s_hi < STORE_PRECOPY * nbk);
    {
        const int nxt = h->cur ^ 1;
        if (store_full || precopy) {
            const int64_t cap = std::max<int64_t>(std::max<int64_t>(h->s_cap, 2 * m_new + m_new / 2 + nbk + 1024),
                                                  steady_store_cap(h, m_new, nbk));
            const void *was = h->st_ts[nxt].p;
            if ((rc = ensure(h, h->st_src[nxt], sizeof(int32_t) * (size_t)cap, true))) return rc;
            if ((rc = ensure(h, h->st_dst[nxt], sizeof(int32_t) * (size_t)cap, true))) return rc;
            if ((rc = ensure(h, h->st_ts[nxt], sizeof(int64_t) * (size_t)cap, true))) return rc;
            if (h->st_ts[nxt].p != was) h->smir_on = false;  // a new buffer holds no copy
        } else if (!append) {
            const int64_t cap =
                std::max<int64_t>(std::max<int64_t>(h->s_cap, 2 * m_new + 1024), steady_store_cap(h, m_new, nbk));
            if ((rc = ensure(h, h->st_src[nxt], sizeof(int32_t) * (size_t)cap))) return rc;
            if ((rc = ensure(h, h->st_dst[nxt], sizeof(int32_t) * (size_t)cap))) return rc;
            if ((rc = ensure(h, h->st_ts[nxt], sizeof(int64_t) * (size_t)cap))) return rc;
        }
        if (ts_full) {
            if ((rc = ensure(h, h->tg, sizeof(int32_t) * (size_t)(2 * m_new + 1024), true))) return rc;
        } else if (ts_move || ts_precopy) {
            const int64_t live = h->tg_hi - h->tg_lo + 1;
            const int64_t tcap = std::max<int64_t>(2 * (live + nbk) + 1024, steady_store_cap(h, m_new, nbk));
            const void *was = h->tg2.p;
            if ((rc = ensure(h, h->tg2, sizeof(int32_t) * (size_t)tcap, true))) return rc;
            if (h->tg2.p != was) h->tmir_on = false;  // a new buffer holds no copy
        }
        if (!nv_full && (rc = nv_prepare_append(h, i0, nbk, N_old, N_new))) return rc;
    }

    // 5. store (from here on a failure is undone by the caller)
    stage.next("ingest: store");
    *changing = true;
    int64_t new_lo = 0;  // first appended index
    bool store_fused = false;  // the batch statistics already wrote the appended edges
    int64_t store_moved = 0;   // live edges copied to the other buffer by this batch
    if (append) {
        // absolute positions of the kept range (after this batch's eviction)
        const int64_t A_lo = h->s_base + h->s_lo + i0, A_hi = h->s_base + h->s_hi;
        const int nxt = h->cur ^ 1;
        // copies the absolute positions [a, b) of the current buffer to the
        // other one, position p at index p - base
        auto copy_out = [&](int64_t a, int64_t b, int64_t base) {
            if (b <= a) return;
            const int64_t from = a - h->s_base, to = a - base, k = b - a;
            cudaMemcpyAsync(h->st_src[nxt].as<int32_t>() + to, h->st_src[h->cur].as<int32_t>() + from,
                            sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(h->st_dst[nxt].as<int32_t>() + to, h->st_dst[h->cur].as<int32_t>() + from,
                            sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(h->st_ts[nxt].as<int64_t>() + to, h->st_ts[h->cur].as<int64_t>() + from,
                            sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToDevice, st);
            store_moved += k;
        };
        if (store_full) {
            // move the kept range to the other buffer: what the pre-copy
            // already holds stays where it is, the rest is copied now
            const int64_t ncap = std::min({(int64_t)(h->st_src[nxt].bytes / 4), (int64_t)(h->st_dst[nxt].bytes / 4),
                                           (int64_t)(h->st_ts[nxt].bytes / 8)});
            const bool held = h->smir_on && h->smir_a0 <= A_lo && A_hi - h->smir_a0 + nbk <= ncap;
            const int64_t base = held ? h->smir_a0 : A_lo;
            copy_out(held ? std::max(h->smir_done, A_lo) : A_lo, A_hi, base);
            h->s_base = base;
            h->cur = nxt;
            h->s_cap = ncap;
            h->s_lo = A_lo - base;
            h->s_hi = A_hi - base;
            h->smir_on = false;
        } else {
            h->s_lo += i0;
            if (precopy) {
                // a share of the rest, so that the copy catches up with the
                // end by the time the buffer fills (appends that still fit,
                // this one included).  It starts where the live range will
                // start then, predicted from this batch's eviction with one
                // batch of margin (the edges evicted before the move are not
                // copied; a move whose live range starts earlier copies it
                // all)
                const int64_t fits = std::max<int64_t>(1, (h->s_cap - h->s_hi) / nbk);
                if (!h->smir_on) {
                    h->smir_on = true;
                    h->smir_a0 = std::min(A_hi, A_lo + std::max<int64_t>(0, fits - 1) * i0);
                    h->smir_done = h->smir_a0;
                }
                const int64_t from = std::max(h->smir_done, A_lo), rest = A_hi - from;
                const int64_t share = (rest + fits - 1) / fits;
                copy_out(from, from + share, h->smir_a0);
                h->smir_done = from + share;
            }
        }
        new_lo = h->s_hi;
        store_fused = spec && sorted && late == 0 && j0 == 0 && old_buf == h->cur && h->s_hi == spec_at;
        if (nbk > 0 && !store_fused) {
            int32_t *os = h->st_src[h->cur].as<int32_t>() + h->s_hi;
            int32_t *od = h->st_dst[h->cur].as<int32_t>() + h->s_hi;
            int64_t *ot = h->st_ts[h->cur].as<int64_t>() + h->s_hi;
            cudaMemcpyAsync(os, bs + j0, sizeof(int32_t) * (size_t)nbk, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(od, bd + j0, sizeof(int32_t) * (size_t)nbk, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(ot, bt + j0, sizeof(int64_t) * (size_t)nbk, cudaMemcpyDeviceToDevice, st);
        }
        h->s_hi += nbk;
    } else {
        const int nxt = h->cur ^ 1;
        h->smir_on = false;  // the merge writes the other buffer
        const int64_t cap =
            std::max<int64_t>(std::max<int64_t>(h->s_cap, 2 * m_new + 1024), steady_store_cap(h, m_new, nbk));
        if ((rc = ensure(h, h->st_src[nxt], sizeof(int32_t) * (size_t)cap))) return rc;
        if ((rc = ensure(h, h->st_dst[nxt], sizeof(int32_t) * (size_t)cap))) return rc;
        if ((rc = ensure(h, h->st_ts[nxt], sizeof(int64_t) * (size_t)cap))) return rc;
        const int64_t a = h->s_lo + i0;
        const int64_t threads = (m_new + MERGE_K - 1) / MERGE_K;
        k_merge<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
            h->st_src[h->cur].as<int32_t>() + a, h->st_dst[h->cur].as<int32_t>() + a, h->st_ts[h->cur].as<int64_t>() + a,
            na, bs + j0, bd + j0, bt + j0, nbk, h->st_src[nxt].as<int32_t>(), h->st_dst[nxt].as<int32_t>(),
            h->st_ts[nxt].as<int64_t>());
        h->pending_launches++;
        h->s_base += h->s_hi;  // every slot is rebuilt below
        h->cur = nxt;
        h->s_cap = std::min({(int64_t)(h->st_src[nxt].bytes / 4), (int64_t)(h->st_dst[nxt].bytes / 4),
                             (int64_t)(h->st_ts[nxt].bytes / 8)});
        h->s_lo = 0;
        h->s_hi = m_new;
    }
    if ((rc = cuda_check(h, cudaGetLastError(), "store"))) return rc;

    // commit the store counters
    h->m = m_new;
    h->N = N_new;
    h->seq_next += n;
    h->dropped += late;
    h->evicted += i0 + j0;
    const int64_t evicted_now = i0 + j0;
    h->has_cutoff = hs->has_cut;
    h->cutoff = hs->cut;

    // 6. timestamp view
    stage.next("ingest: timestamp view");
    int64_t ts_moved = 0;
    // copies the starts [a, b) of tg to tg2 at index position - base
    auto tg_copy = [&](int64_t a, int64_t b, int64_t base) {
        if (b <= a) return;
        cudaMemcpyAsync(h->tg2.as<int32_t>() + (a - base), h->tg.as<int32_t>() + a, sizeof(int32_t) * (size_t)(b - a),
                        cudaMemcpyDeviceToDevice, st);
        ts_moved += b - a;
    };
    if (ts_full) {
        h->tmir_on = false;
    } else if (ts_move) {
        // move the live starts [tg_lo, tg_hi] to a larger buffer: what the
        // copy made ahead holds stays where it is, the rest is copied now
        const int64_t ncap = (int64_t)(h->tg2.bytes / sizeof(int32_t));
        const bool held = h->tmir_on && h->tmir_a0 <= h->tg_lo && h->tg_hi - h->tmir_a0 + nbk + 2 <= ncap;
        const int64_t base = held ? h->tmir_a0 : h->tg_lo;
        tg_copy(held ? std::max(h->tmir_done, h->tg_lo) : h->tg_lo, h->tg_hi + 1, base);
        std::swap(h->tg, h->tg2);
        h->tg_hi -= base;
        h->tg_lo -= base;
        h->tmir_on = false;
    } else if (ts_precopy) {
        // a share of the starts before the tail entry (the batch overwrites
        // that one), from the predicted first live group at the move
        const int64_t fits = std::max<int64_t>(1, tg_room / nbk);
        if (!h->tmir_on) {
            h->tmir_on = true;
            h->tmir_a0 = std::min(h->tg_hi, h->tg_lo + std::max<int64_t>(0, fits - 1) * h->tg_lo_step);
            h->tmir_done = h->tmir_a0;
        }
        const int64_t from = std::max(h->tmir_done, h->tg_lo), rest = h->tg_hi - from;
        const int64_t share = (rest + fits - 1) / fits;
        tg_copy(from, from + share, h->tmir_a0);
        h->tmir_done = from + share;
    }
    if (ts_full) {
        if ((rc = ts_view_build(h))) return rc;
    } else {
        k_ts_evict<<<1, 32, 0, st>>>(h->tg.as<int32_t>(), h->tg_lo, h->tg_hi, abs32(h, h->s_lo), ds);
        int nbl;
        if (sorted) {
            // the kept edges are the batch's edges late + j0 onwards, in order
            const uint8_t *f0 = h->b_gflag.as<uint8_t>() + late + j0;
            const int64_t a = (int64_t)((uintptr_t)f0 & 15);
            TsTailBytes op{f0 - a, a, nbk, h->st_ts[h->cur].as<int64_t>(), new_lo, h->s_lo, abs32(h, 0),
                           h->tg.as<int32_t>() + h->tg_hi};
            nbl = bscan_launch(op, h->partials.as<uint64_t>(), st);
        } else {
            TsGroupOp op{h->st_ts[h->cur].as<int64_t>(), new_lo, h->s_lo, abs32(h, 0),
                         h->tg.as<int32_t>() + h->tg_hi};
            nbl = scan_launch(op, nbk, h->partials.as<uint64_t>(), st);
        }
        k_ts_tail<<<1, 1, 0, st>>>(h->tg.as<int32_t>(), h->tg_hi, h->partials.as<uint64_t>() + nbl,
                                   abs32(h, h->s_hi), ds);
        h->pending_launches += 5;
    }

    // 7. node view
    stage.next("ingest: node view");
    bool nv_pending = false;
    if (!nv_full) {
        rc = nv_append(h, h->st_src[old_buf].as<int32_t>() + old_lo, h->st_dst[old_buf].as<int32_t>() + old_lo, i0,
                       new_lo, nbk, N_old);
        if (rc) return rc;
        nv_pending = true;  // finished after the round trip below
    } else if ((rc = nv_build(h))) {
        return rc;
    }

    stage.next("ingest: pair table");
    // 8. Node2Vec pair table: the evicted edges out, the kept batch in (a
    // rebuild after a merge, whose evicted edges are not a store range)
    if (h->pt_on) {
        rc = append ? pt_update(h, h->st_src[old_buf].as<int32_t>() + old_lo,
                                h->st_dst[old_buf].as<int32_t>() + old_lo, i0, new_lo, nbk, &ds->status)
                    : pt_rebuild(h, &ds->status);
        if (rc) return rc;  // undone by the caller, which rebuilds the table from the restored store
    }

    cudaMemcpyAsync(hs, ds, sizeof(IngestScratch), cudaMemcpyDeviceToHost, st);
    // the node view's counters in the same round trip (their own pinned slot)
    NvCounters *hn = reinterpret_cast<NvCounters *>(static_cast<char *>(h->hstat) + 1024);
    if (nv_pending) cudaMemcpyAsync(hn, h->nvc.p, sizeof(NvCounters), cudaMemcpyDeviceToHost, st);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "ingest"))) return rc;
    if (hs->status)
        return fail(h, TEMPEST_ECUDA, "ingest: index consistency check failed (code 0x%llx)",
                    (unsigned long long)hs->status);
    if (nv_pending) {
        bool rebuild = false;
        if ((rc = nv_append_finish(h, hn, &rebuild))) return rc;
        if (rebuild) {
            nv_full = true;
            if ((rc = nv_build(h))) return rc;
        }
    }
    const int64_t tg_added_now = (int64_t)hs->tg_added;
    if (ts_full) {
        h->tg_lo = 0;
        h->tg_hi = hs->tg_added;
        h->tg_lo_step = 0;
    } else {
        h->tg_lo_step = hs->tg_lo - h->tg_lo;
        h->tg_lo = hs->tg_lo;
        h->tg_hi += hs->tg_added;
    }
    h->G = h->tg_hi - h->tg_lo;

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
        float ms = 0.f;
        // the events ran before the sync above; a rebuild after the append
        // makes the batch's eviction part of the rebuild
        stats->evict_ms = (h->eev_valid && !nv_full && cudaEventElapsedTime(&ms, h->eev[0], h->eev[1]) == cudaSuccess)
                              ? (double)ms : 0.0;
        const int ts_passes = sorted ? 0 : (bits_for(span) + RADIX_BITS - 1) / RADIX_BITS;
        stats->model_bytes = ingest_model_bytes(h->nv_rep, n, nbk, na, m_new, ts_passes, append, store_fused,
                                                ts_full, tg_added_now, h->G, store_moved, ts_moved);
        stats->view_rebuilt = h->nv_rep.rebuilt ? 1 : 0;
        stats->copied_ahead = (int32_t)h->nv_rep.copied_ahead;
    }
    return TEMPEST_OK;
}

}  // namespace tw
