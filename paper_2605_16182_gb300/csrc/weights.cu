// weights.cu -- per-group weights and per-node suffix sums for the
// weight-based exponential sampler (Tempest Sec. 2.5, the paper's default
// sampler: every edge of Gamma_t(v) weighs exp(lambda (t_e - t_min)) and the
// next edge is an inverse-CDF draw on the running weight).
//
// Edges of one (node, timestamp) group weigh the same, so the draw picks a
// group by the groups' weights (size * exp(lambda t)) and then an edge of it
// uniformly (the paper's uniform tie rule).  Any per-node reference time
// gives the same distribution, so each node keeps one, wref[v], and its
// groups' weights gw[g] = size_g * exp(lambda (t_g - wref[v])) are computed
// once, when a batch creates or grows the group.  A node's reference moves
// (all weights recomputed) only when a new group's exponent exceeds
// W_REBASE, when the rate changes, and after a full rebuild of the view.
//
// For the walks of an index state, each node's suffix sums
// gs[g] = sum of gw over [g, g_hi) are built by a segmented reverse scan in
// three passes over 1024-group chunks: chunk totals, per-node suffix offsets
// of the chunk totals, then the chunk-local reverse scan plus its offset.
// A hop at node v with Gamma = groups [c, g1) then needs gs[c] (the weight
// of Gamma, with no cancellation: Gamma is a suffix) and the smallest k with
// gs[k + 1] <= gs[c] (1 - u): the group whose running weight from c first
// reaches u gs[c].
#include <algorithm>

#include "engine.cuh"
#include "prims.cuh"
#include "sortscan.cuh"

namespace tw {

namespace {

constexpr int WCH = 1024;           // groups per chunk
constexpr double W_REBASE = 600.0;  // exponent above which a node's reference moves

struct WChunkOp {
    const int32_t *act;
    const NodeRange *ngr;
    int32_t *cbase;
    __device__ __forceinline__ uint64_t value(int64_t j) const
    {
        const NodeRange &r = ngr[act[j]];
        return (uint64_t)((r.g_hi - r.g_lo + WCH - 1) / WCH);
    }
    __device__ __forceinline__ void emit(int64_t j, uint64_t, uint64_t ex) const { cbase[j] = (int32_t)ex; }
};

__global__ void k_w_tail(int32_t *cbase, int64_t n, const uint64_t *tot) { cbase[n] = (int32_t)*tot; }

// Index of the node (in act) owning chunk c: the last j with cbase[j] <= c
// (nodes without groups own no chunk and share the next node's base).
__device__ __forceinline__ int64_t chunk_owner(const int32_t *__restrict__ cbase, int64_t n, int64_t c)
{
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(cbase + mid) <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double group_weight(int32_t size, int64_t t, int64_t ref, double lam)
{
    return (double)size * exp(lam * (double)(t - ref));
}

// Every live group of every node: the reference becomes the node's newest
// group time (weights <= size).  One warp per chunk.
__global__ void __launch_bounds__(256) k_w_all(const int32_t *__restrict__ act, int64_t n_act,
                                               const int32_t *__restrict__ cbase, const NodeRange *__restrict__ ngr,
                                               const int32_t *__restrict__ ngo, const int64_t *__restrict__ ngts,
                                               double lam, int64_t *wref, double *gw)
{
    const int lane = threadIdx.x & 31;
    const int64_t nch = cbase[n_act];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += warps) {
        const int64_t j = chunk_owner(cbase, n_act, c);
        const int32_t v = act[j];
        const NodeRange r = ngr[v];
        if (c == cbase[j] && lane == 0) wref[v] = r.t_last;
        const int32_t a = r.g_lo + (int32_t)(c - cbase[j]) * WCH;
        const int32_t b = min(r.g_hi, a + WCH);
        for (int32_t g = a + lane; g < b; g += 32)
            gw[g] = group_weight(ngo[g + 1] - ngo[g], ngts[g], r.t_last, lam);
    }
}

// Groups the batch created (a flagged entry starts one) or grew (a run whose
// first entry joined the node's last group): their weights.  A node without
// live groups before the batch takes its first new group's time as
// reference.  Runs after the scatter of the batch (ngo holds the new ends);
// one block per tile of the batch's entries, whose runs and groups come from
// the flag bytes (RunTile).
__global__ void __launch_bounds__(BSCAN_THREADS)
    k_w_append(const uint8_t *__restrict__ flags, int64_t nbe, const uint64_t *__restrict__ tile_prefix,
               const int32_t *__restrict__ run_g, const int32_t *__restrict__ run_dg,
               const int32_t *__restrict__ run_node, const NodeRange *__restrict__ ngr, const int32_t *__restrict__ ngo,
               const int64_t *__restrict__ ngts, double lam, int64_t *wref, double *gw, NvCounters *cnt)
{
    if (cnt->overflow) return;  // the batch rebuilds the view (and the weights) instead
    __shared__ RunTile sm;
    const int64_t t = blockIdx.x, p0 = t * BSCAN_TILE;
    run_tile_load(sm, flags, nbe, t, tile_prefix[t]);
    for (int k = 0; k < 16; k++) {
        const int j = k * BSCAN_THREADS + threadIdx.x;
        if (p0 + j >= nbe) break;
        const RunAt a = run_tile_at(sm, j);
        const bool opens = a.gs, first = a.rs;
        if (!opens && !first) continue;
        const int32_t r = a.r;
        const int32_t v = run_node[r];
        const int32_t dg = run_dg[r];
        const bool was_empty = ngr[v].g_lo == dg;
        const int64_t ref = was_empty ? ngts[dg] : wref[v];
        if (first && was_empty) wref[v] = ref;
        const int32_t g = opens ? dg + (a.g - run_g[r]) : dg - 1;  // else: the grown last group
        const double e = lam * (double)(ngts[g] - ref);
        if (e > W_REBASE) atomicOr(&cnt->w_rebase, 1ull);
        gw[g] = (double)(ngo[g + 1] - ngo[g]) * exp(e);
    }
}

// Sum of the weights of each chunk.
__global__ void __launch_bounds__(256) k_w_ctot(const int32_t *__restrict__ act, int64_t n_act,
                                                const int32_t *__restrict__ cbase,
                                                const NodeRange *__restrict__ ngr, const double *__restrict__ gw,
                                                double *ctot)
{
    const int lane = threadIdx.x & 31;
    const int64_t nch = cbase[n_act];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += warps) {
        const int64_t j = chunk_owner(cbase, n_act, c);
        const NodeRange r = ngr[act[j]];
        const int32_t a = r.g_lo + (int32_t)(c - cbase[j]) * WCH;
        const int32_t b = min(r.g_hi, a + WCH);
        double s = 0.0;
        for (int32_t g = a + lane; g < b; g += 32) s += gw[g];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) ctot[c] = s;
    }
}

// Per node: the weight of its chunks after each chunk (one warp per node,
// from the last chunk backwards, 32 chunks per step).
__global__ void __launch_bounds__(256) k_w_coff(const int32_t *__restrict__ cbase, int64_t n_act,
                                                const double *__restrict__ ctot, double *coff)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n_act; j += warps) {
        const int64_t c0 = cbase[j], c1 = cbase[j + 1];
        double carry = 0.0;
        for (int64_t top = c1; top > c0; top -= 32) {
            const int64_t c = top - 1 - lane;  // lane 0 takes the last chunk of the step
            const double x = c >= c0 ? ctot[c] : 0.0;
            // inclusive sum over this lane and the lanes before it (later chunks)
            double s = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            if (c >= c0) coff[c] = carry + s - x;
            carry += __shfl_sync(0xffffffffu, s, 31);
        }
    }
}

// Suffix sums inside each chunk plus the chunk's offset; the node's last
// chunk also closes the node with gs[g_hi] = 0.
__global__ void __launch_bounds__(256) k_w_suffix(const int32_t *__restrict__ act, int64_t n_act,
                                                  const int32_t *__restrict__ cbase,
                                                  const NodeRange *__restrict__ ngr, const double *__restrict__ gw,
                                                  const double *__restrict__ coff, double *gs)
{
    const int lane = threadIdx.x & 31;
    const int64_t nch = cbase[n_act];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += warps) {
        const int64_t j = chunk_owner(cbase, n_act, c);
        const NodeRange r = ngr[act[j]];
        const int32_t a = r.g_lo + (int32_t)(c - cbase[j]) * WCH;
        const int32_t b = min(r.g_hi, a + WCH);
        if (b == r.g_hi && lane == 0) gs[b] = 0.0;
        double carry = coff[c];
        // 32-group steps from the end of the chunk; within a step a reverse
        // inclusive scan over the lanes
        const int32_t steps = (b - a + 31) / 32;
        for (int32_t k = steps - 1; k >= 0; k--) {
            const int32_t g = a + 32 * k + lane;
            const double x = g < b ? gw[g] : 0.0;
            double s = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_down_sync(0xffffffffu, s, o);
                if (lane + o < 32) s += y;
            }
            if (g < b) gs[g] = carry + s;
            carry += __shfl_sync(0xffffffffu, s, 0);
        }
    }
}

unsigned wgrid(tempest_t *h, int64_t items)
{
    int64_t g = (items + 7) / 8;
    const int64_t cap = (int64_t)h->num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// Chunk list of the nodes owning regions; returns the chunk count.
int w_chunks(tempest_t *h, int64_t &nch)
{
    cudaStream_t st = h->stream;
    int rc;
    const int64_t n = h->n_act;
    if ((rc = ensure(h, h->w_cbase, sizeof(int32_t) * (size_t)(n + 1), true))) return rc;
    WChunkOp op{h->act.as<int32_t>(), h->ngr.as<NodeRange>(), h->w_cbase.as<int32_t>()};
    uint64_t *part = h->partials.as<uint64_t>();
    const int nb = scan_launch(op, n, part, st);
    k_w_tail<<<1, 1, 0, st>>>(h->w_cbase.as<int32_t>(), n, part + nb);
    uint64_t *hp = static_cast<uint64_t *>(h->hstat);
    cudaMemcpyAsync(hp, part + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "weight chunks"))) return rc;
    nch = (int64_t)hp[0];
    return TEMPEST_OK;
}

int ensure_weight_pools(tempest_t *h)
{
    int rc;
    const size_t gz = (size_t)(h->g_cap > 0 ? h->g_cap : 1);
    if ((rc = ensure(h, h->gw, sizeof(double) * gz))) return rc;
    if ((rc = ensure(h, h->gs, sizeof(double) * gz))) return rc;
    if ((rc = ensure(h, h->wref, sizeof(int64_t) * (size_t)(h->nrec_n > 0 ? h->nrec_n : 1)))) return rc;
    return TEMPEST_OK;
}

}  // namespace

int nv_append_weights(tempest_t *h, int64_t nbe)
{
    if (!h->w_on || !h->w_valid || nbe <= 0) return TEMPEST_OK;
    // pools that would have to grow lose their contents: recompute all later
    if (h->gw.bytes < sizeof(double) * (size_t)h->g_cap || h->gs.bytes < sizeof(double) * (size_t)h->g_cap ||
        h->wref.bytes < sizeof(int64_t) * (size_t)h->nrec_n) {
        h->w_valid = false;
        return TEMPEST_OK;
    }
    cudaStream_t st = h->stream;
    const unsigned grid = (unsigned)((nbe + BSCAN_TILE - 1) / BSCAN_TILE);
    k_w_append<<<grid, BSCAN_THREADS, 0, st>>>(h->nv_flags.as<uint8_t>(), nbe, h->nv_tex.as<uint64_t>(),
                                               h->run_g.as<int32_t>(), h->run_dg.as<int32_t>(),
                                               h->run_node.as<int32_t>(), h->ngr.as<NodeRange>(),
                                               h->ngo.as<int32_t>(), h->ngts.as<int64_t>(), h->lam_w,
                                               h->wref.as<int64_t>(), h->gw.as<double>(), h->nvc.as<NvCounters>());
    h->pending_launches++;
    return cuda_check(h, cudaGetLastError(), "append weights");
}

int prepare_weights(tempest_t *h)
{
    int rc;
    if (!h->w_on) {
        h->w_on = true;
        h->w_valid = false;
    }
    if (h->w_valid && h->w_ver == h->state_ver) return TEMPEST_OK;
    cudaStream_t st = h->stream;
    if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
    if (h->n_act <= 0 || h->Gn <= 0 || !h->nv_ready) {
        h->w_valid = true;
        h->w_ver = h->state_ver;
        return TEMPEST_OK;
    }
    if ((rc = ensure_weight_pools(h))) return rc;
    int64_t nch = 0;
    if ((rc = w_chunks(h, nch))) return rc;
    const int32_t *act = h->act.as<int32_t>();
    const int32_t *cb = h->w_cbase.as<int32_t>();
    const NodeRange *ngr = h->ngr.as<NodeRange>();
    if (!h->w_valid) {
        k_w_all<<<wgrid(h, nch), 256, 0, st>>>(act, h->n_act, cb, ngr, h->ngo.as<int32_t>(), h->ngts.as<int64_t>(),
                                                h->lam_w, h->wref.as<int64_t>(), h->gw.as<double>());
        h->w_valid = true;
    }
    if ((rc = ensure(h, h->w_ctot, sizeof(double) * (size_t)(nch > 0 ? nch : 1), true))) return rc;
    if ((rc = ensure(h, h->w_coff, sizeof(double) * (size_t)(nch > 0 ? nch : 1), true))) return rc;
    k_w_ctot<<<wgrid(h, nch), 256, 0, st>>>(act, h->n_act, cb, ngr, h->gw.as<double>(), h->w_ctot.as<double>());
    k_w_coff<<<wgrid(h, h->n_act), 256, 0, st>>>(cb, h->n_act, h->w_ctot.as<double>(), h->w_coff.as<double>());
    k_w_suffix<<<wgrid(h, nch), 256, 0, st>>>(act, h->n_act, cb, ngr, h->gw.as<double>(), h->w_coff.as<double>(),
                                               h->gs.as<double>());
    if ((rc = cuda_check(h, cudaGetLastError(), "weight suffix sums"))) return rc;
    h->w_ver = h->state_ver;
    return TEMPEST_OK;
}

}  // namespace tw

extern "C" int tempest_set_weight_rate(tempest_t *h, double lambda_w)
{
    if (!h) return TEMPEST_EINVAL;
    if (!(lambda_w > 0.0) || !(lambda_w < 1e300))
        return tw::fail(h, TEMPEST_EINVAL, "tempest_set_weight_rate: lambda_w must be positive and finite");
    h->lam_w = lambda_w;
    h->w_on = true;
    h->w_valid = false;
    return TEMPEST_OK;
}
