// pairs.cu -- the live-pair table of Temporal Node2Vec (Sec. 2.5).
//
// A Node2Vec hop from node v, reached from u, weighs a candidate w by 1 when
// w is a neighbour of u: when the window holds a live edge u -> w (either
// orientation for undirected graphs).  The table answers that test with one
// or two 16-byte probes: open addressing with linear probing over PairSlot
// {key, count}, key = from << 32 | to (the smaller id first for undirected
// graphs), count = live edges with that key.
//
// Ingest keeps it current in work proportional to the batch: the evicted
// edges' counts are decremented and the batch's kept edges inserted or
// incremented (atomics; the probe sequence of a key is fixed, so concurrent
// inserts of one key meet in one slot).  A key whose count reaches 0 keeps its
// slot until the next rebuild, so the host tracks an upper bound of used
// slots and rebuilds from the live store when it would pass half the
// capacity (and after out-of-order merges, where the evicted edges are not a
// store range).  Capacity: the power of two >= 4 x the live edges, so a
// rebuild happens every (capacity / 2 - m) / b batches of b edges.
#include <algorithm>

#include "engine.cuh"
#include "walkcore.cuh"

namespace tw {

namespace {

__global__ void k_pt_clear(PairSlot *t, int64_t cap)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = PairSlot{PAIR_EMPTY, 0, 0};
}

// delta = +1: insert (or count) every pair; -1: uncount every pair (each must
// be present).  Lanes of a warp holding the same key combine first (a Zipf
// stream repeats its hub pairs in every warp), so a key takes one atomic per
// warp.  A probe sequence longer than the table sets a status bit.
__global__ void k_pt_apply(PairSlot *t, uint64_t mask, const int32_t *__restrict__ a, const int32_t *__restrict__ b,
                           int64_t n, int directed, int delta, unsigned long long *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < n;
        const unsigned long long key = valid ? pair_key(a[i], b[i], directed) : PAIR_EMPTY;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (!valid || lane != __ffs(peers) - 1) continue;
        const int d = delta * __popc(peers);
        uint64_t s = pair_hash(key) & mask;
        bool done = false;
        for (uint64_t probe = 0; probe <= mask && !done; probe++, s = (s + 1) & mask) {
            unsigned long long k = t[s].key;
            if (k == PAIR_EMPTY && delta > 0) k = atomicCAS(&t[s].key, PAIR_EMPTY, key);
            if (k == PAIR_EMPTY && delta > 0) k = key;  // this thread claimed the slot
            if (k == key) {
                atomicAdd(&t[s].cnt, d);
                done = true;
            } else if (k == PAIR_EMPTY) {
                break;  // a decrement of an absent key
            }
        }
        if (!done) atomicOr(status, 1ull << 16);
    }
}

int64_t grid_of(const tempest_t *h, int64_t n)
{
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)h->num_sms * 16;
    return std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

// Rebuilds the table from the live store, sized for it.
int pt_rebuild(tempest_t *h, unsigned long long *status)
{
    int64_t cap = 1024;
    while (cap < 4 * h->m) cap <<= 1;
    int rc;
    if ((rc = ensure(h, h->pt, sizeof(PairSlot) * (size_t)cap, true))) return rc;
    h->pt_cap = cap;
    cudaStream_t st = h->stream;
    k_pt_clear<<<(unsigned)grid_of(h, cap), 256, 0, st>>>(h->pt.as<PairSlot>(), cap);
    if (h->m > 0)
        k_pt_apply<<<(unsigned)grid_of(h, h->m), 256, 0, st>>>(
            h->pt.as<PairSlot>(), (uint64_t)cap - 1, h->st_src[h->cur].as<int32_t>() + h->s_lo,
            h->st_dst[h->cur].as<int32_t>() + h->s_lo, h->m, h->directed, 1, status);
    h->pt_ub = h->m;
    h->pending_launches += h->m > 0 ? 2 : 1;
    return cuda_check(h, cudaGetLastError(), "pair table rebuild");
}

// After a batch appended at the store's tail: the evicted edges (ev_*, n_ev,
// still readable in the buffer they left) are uncounted and the kept batch
// edges (store indices [add_lo, add_lo + n_add) of the current buffer)
// counted; a rebuild instead when the used-slot bound would pass half the
// capacity.
int pt_update(tempest_t *h, const int32_t *ev_src, const int32_t *ev_dst, int64_t n_ev, int64_t add_lo,
              int64_t n_add, unsigned long long *status)
{
    if (!h->pt.p || 2 * (h->pt_ub + n_add) > h->pt_cap) return pt_rebuild(h, status);
    cudaStream_t st = h->stream;
    const uint64_t mask = (uint64_t)h->pt_cap - 1;
    if (n_ev > 0) {
        k_pt_apply<<<(unsigned)grid_of(h, n_ev), 256, 0, st>>>(h->pt.as<PairSlot>(), mask, ev_src, ev_dst, n_ev,
                                                               h->directed, -1, status);
        h->pending_launches++;
    }
    if (n_add > 0) {
        k_pt_apply<<<(unsigned)grid_of(h, n_add), 256, 0, st>>>(
            h->pt.as<PairSlot>(), mask, h->st_src[h->cur].as<int32_t>() + add_lo,
            h->st_dst[h->cur].as<int32_t>() + add_lo, n_add, h->directed, 1, status);
        h->pending_launches++;
    }
    h->pt_ub += n_add;
    return cuda_check(h, cudaGetLastError(), "pair table update");
}

}  // namespace tw

using namespace tw;

extern "C" int tempest_set_node2vec(tempest_t *h, double p, double q)
{
    if (!h) return TEMPEST_EINVAL;
    if (!(p >= 1e-3 && p <= 1e3) || !(q >= 1e-3 && q <= 1e3))
        return fail(h, TEMPEST_EINVAL, "tempest_set_node2vec: p and q must lie in [1e-3, 1e3]");
    h->n2v_p = p;
    h->n2v_q = q;
    if (q == 1.0 || h->pt_on) return TEMPEST_OK;  // q = 1: the neighbour test never changes a weight
    // from now on ingest keeps the table of live pairs
    int rc;
    if ((rc = ensure(h, h->dstat, sizeof(IngestScratch)))) return rc;
    IngestScratch *ds = h->dstat.as<IngestScratch>();
    cudaMemsetAsync(&ds->status, 0, sizeof(ds->status), h->stream);
    if ((rc = pt_rebuild(h, &ds->status))) return rc;
    unsigned long long hs = 0;
    cudaMemcpyAsync(&hs, &ds->status, sizeof(hs), cudaMemcpyDeviceToHost, h->stream);
    if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "tempest_set_node2vec"))) return rc;
    if (hs) return fail(h, TEMPEST_ECUDA, "tempest_set_node2vec: pair table check failed (0x%llx)", hs);
    h->pt_on = true;
    return TEMPEST_OK;
}
