// capi.cu -- the extern "C" entry points declared in include/tempest.h, and
// the handle's memory management.
#include <sched.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "engine.cuh"
#include "prims.cuh"
#include "sortscan.cuh"

namespace tw {

__global__ void k_scan_partials(uint64_t *p, int nb)
{
    __shared__ uint64_t sh[33];
    uint64_t carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint64_t v = i < nb ? p[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_scan<uint64_t>(v, sh, tot);
        if (i < nb) p[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) p[nb] = carry;
}

static thread_local std::string g_create_err;

int fail(tempest_t *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_err = buf;
    return code;
}

int cuda_check(tempest_t *h, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return TEMPEST_OK;
    cudaGetLastError();
    return fail(h, TEMPEST_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void release(tempest_t *h, DBuf &b)
{
    if (!b.p) return;
    if (h->release_fn) h->release_fn(b.p, h->alloc_ctx);
    else cudaFree(b.p);
    h->in_use -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

// Make b hold at least `bytes`.  Contents are not preserved.  With headroom
// the buffer grows by 25 % beyond the request so that a slowly growing
// window does not reallocate on every batch.
int ensure(tempest_t *h, DBuf &b, size_t bytes, bool headroom)
{
    if (bytes == 0) bytes = 1;
    if (b.p && b.bytes >= bytes) return TEMPEST_OK;
    size_t want = bytes;
    if (headroom && b.p) want = bytes + bytes / 4;
    want = (want + 255) & ~(size_t)255;
    if (h->budget && h->in_use - b.bytes + want > h->budget) {
        want = (bytes + 255) & ~(size_t)255;
        if (h->in_use - b.bytes + want > h->budget)
            return fail(h, TEMPEST_ENOMEM, "HBM budget of %zu bytes exceeded (in use %zu, need %zu more)",
                        h->budget, h->in_use - b.bytes, want);
    }
    release(h, b);
    void *p = nullptr;
    if (h->alloc_fn) {
        p = h->alloc_fn(want, h->alloc_ctx);
        if (!p) return fail(h, TEMPEST_ENOMEM, "allocator callback returned NULL for %zu bytes", want);
        if ((uintptr_t)p & 255) {  // kernels load 16-byte records and vectors from every buffer
            if (h->release_fn) h->release_fn(p, h->alloc_ctx);
            else cudaFree(p);
            return fail(h, TEMPEST_EINVAL, "allocator callback returned %p, not 256-byte aligned", p);
        }
    } else {
        const cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, TEMPEST_ENOMEM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
        }
    }
    b.p = p;
    b.bytes = want;
    h->in_use += want;
    return TEMPEST_OK;
}

// Offsets of the walks' cells in the compacted copy (exclusive prefix of the
// lengths, each clamped to the row).
struct LenScanOp {
    const int32_t *len;
    int32_t cap;
    int64_t *off;
    __device__ __forceinline__ uint64_t value(int64_t i) const
    {
        const int32_t l = len[i];
        return (uint64_t)(l < 0 ? 0 : (l > cap ? cap : l));
    }
    __device__ __forceinline__ void emit(int64_t i, uint64_t, uint64_t ex) const { off[i] = (int64_t)ex; }
};

// The cells [0, len) of every row, back to back (a thread per walk: walks
// are a few cells long).
__global__ void k_compact_rows(const int32_t *__restrict__ node, const int64_t *__restrict__ ts,
                               const int32_t *__restrict__ len, const int64_t *__restrict__ off, int64_t n,
                               int32_t cap, int32_t *cnode, int64_t *cts)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t l = len[i];
        l = l < 0 ? 0 : (l > cap ? cap : l);
        const int64_t o = off[i];
        const int32_t *nr = node + i * (int64_t)cap;
        const int64_t *tr = ts + i * (int64_t)cap;
        for (int32_t j = 0; j < l; j++) {
            cnode[o + j] = nr[j];
            cts[o + j] = tr[j];
        }
    }
}

// Pinned host staging of at least `bytes` (kept, grown by half again).
// CPUs this process may run on: its affinity mask, capped by a cgroup v2 CPU
// quota ("quota period" in cpu.max) when one is set.  More threads than that
// only time-slice, and past a quota the scheduler stalls them all until its
// next period.
static int host_cpus()
{
    static const int n = [] {
        int c = (int)std::thread::hardware_concurrency();
        cpu_set_t set;
        CPU_ZERO(&set);
        if (sched_getaffinity(0, sizeof(set), &set) == 0 && CPU_COUNT(&set) > 0) c = CPU_COUNT(&set);
        if (FILE *f = fopen("/sys/fs/cgroup/cpu.max", "r")) {
            char q[32] = {0};
            long long per = 0;
            if (fscanf(f, "%31s %lld", q, &per) == 2 && strcmp(q, "max") != 0 && per > 0) {
                const long long quota = atoll(q);
                if (quota > 0) c = std::min<long long>(c, std::max(1LL, quota / per));
            }
            fclose(f);
        }
        return std::max(1, c);
    }();
    return n;
}

static int ensure_pinned(tempest_t *h, size_t bytes)
{
    if (h->hpin_bytes >= bytes) return TEMPEST_OK;
    if (h->hpin) cudaFreeHost(h->hpin);
    h->hpin = nullptr;
    h->hpin_bytes = 0;
    const size_t want = bytes + bytes / 2;
    if (cudaMallocHost(&h->hpin, want) != cudaSuccess) {
        cudaGetLastError();
        h->hpin = nullptr;
        return fail(h, TEMPEST_ENOMEM, "walks: pinned host staging of %zu bytes", want);
    }
    h->hpin_bytes = want;
    return TEMPEST_OK;
}

// Host side of a walk call into host buffers: rows [i0, i1) from the
// compacted cells.  The rows of a range are contiguous, so the range is
// first filled with padding in two long sweeps (node -1 bytewise, ts
// INT64_MIN), then each walk's cells are copied over its row's head.
static void expand_rows(int64_t i0, int64_t i1, int32_t cap, const int32_t *len, const int64_t *off,
                        const int32_t *cnode, const int64_t *cts, int32_t *node, int64_t *ts)
{
    const size_t cells = (size_t)(i1 - i0) * (size_t)cap;
    memset(node + i0 * (int64_t)cap, 0xff, sizeof(int32_t) * cells);
    int64_t *t0 = ts + i0 * (int64_t)cap;
    for (size_t k = 0; k < cells; k++) t0[k] = INT64_MIN;
    for (int64_t i = i0; i < i1; i++) {
        int32_t l = len[i];
        l = l < 0 ? 0 : (l > cap ? cap : l);
        memcpy(node + i * (int64_t)cap, cnode + off[i], sizeof(int32_t) * (size_t)l);
        memcpy(ts + i * (int64_t)cap, cts + off[i], sizeof(int64_t) * (size_t)l);
    }
}

static void free_all(tempest_t *h)
{
    DBuf *bufs[] = {&h->st_src[0], &h->st_src[1], &h->st_dst[0], &h->st_dst[1], &h->st_ts[0], &h->st_ts[1],
                    &h->tg,        &h->ent,       &h->ngo,       &h->ngts,      &h->ngr,       &h->nrec,
                    &h->act,       &h->nvc,       &h->nv_tmp,    &h->run_node,  &h->run_pos,   &h->run_g,
                    &h->run_of,    &h->fx,        &h->run_de,    &h->run_dg,    &h->ev_nodes,  &h->reloc,
                    &h->ev,        &h->b_src,     &h->b_dst,     &h->b_ts,      &h->sb_src,    &h->sb_dst,
                    &h->sb_ts,     &h->sk64[0],   &h->sk64[1],   &h->sk32[0],   &h->sk32[1],   &h->sv[0],
                    &h->sv[1],     &h->hist,      &h->partials,  &h->dstat,     &h->wcnt,      &h->out_stage,
                    &h->in_stage,  &h->exp_stage, &h->co_node,   &h->co_t,      &h->co_len,    &h->co_act[0],
                    &h->co_act[1], &h->co_runs,   &h->co_tasks,  &h->co_ctr,    &h->bkt,
                    &h->big_node,  &h->big_t,     &h->big_c,     &h->tune_out,  &h->dense,     &h->touched,   &h->tg2,       &h->nbeg,
                    &h->pn_nodes,  &h->gw,        &h->gs,        &h->wref,      &h->w_cbase,   &h->w_ctot,
                    &h->w_coff,    &h->co_prev,   &h->pt,        &h->big_own,   &h->big_aux0,
                    &h->big_aux1,  &h->big_bf,    &h->bkt_prev,  &h->nev,       &h->cmp_stage, &h->cmp_off,
                    &h->ent_tmp,   &h->nv_flags,  &h->b_gflag,   &h->nv_tex,    &h->nv_mir};
    for (DBuf *b : bufs) release(h, *b);
}

// Walks per active node of a PER_NODE request (0 for other policies);
// EINVAL when the active nodes do not divide n_walks.
int per_node_k(tempest_t *h, int start_policy, int64_t n_walks, int64_t &k, const char *who)
{
    k = 0;
    if (start_policy != TEMPEST_START_PER_NODE || n_walks == 0) return TEMPEST_OK;
    int rc;
    if ((rc = prepare_active_nodes(h))) return rc;
    if (h->n_pn == 0) {
        k = 1;  // empty window: every walk has length 0
        return TEMPEST_OK;
    }
    if (n_walks % h->n_pn != 0)
        return fail(h, TEMPEST_EINVAL, "%s: PER_NODE needs a multiple of the %lld active nodes, got %lld walks", who,
                    (long long)h->n_pn, (long long)n_walks);
    k = n_walks / h->n_pn;
    return TEMPEST_OK;
}

}  // namespace tw

using namespace tw;

extern "C" {

const char *tempest_version(void) { return "tempest-gb300 0.1 (sm_103a)"; }

const char *tempest_last_error(tempest_t *h)
{
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

int tempest_create(int64_t window, int directed, tempest_t **out)
{
    if (!out) return fail(nullptr, TEMPEST_EINVAL, "tempest_create: out is NULL");
    *out = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, TEMPEST_ECUDA, "tempest_create: no CUDA device: %s", cudaGetErrorString(e));
    }
    tempest_t *h = new (std::nothrow) tempest();
    if (!h) return fail(nullptr, TEMPEST_ENOMEM, "tempest_create: out of host memory");
    h->window = window;
    h->directed = directed ? 1 : 0;
    h->device = dev;
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (h->num_sms < 1) h->num_sms = 1;
    e = cudaMallocHost(&h->hstat, 4096);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, TEMPEST_ENOMEM, "tempest_create: pinned host buffer: %s", cudaGetErrorString(e));
    }
    memset(h->hstat, 0, 4096);
    *out = h;
    return TEMPEST_OK;
}

int tempest_destroy(tempest_t *h)
{
    if (!h) return TEMPEST_OK;
    cudaStreamSynchronize(h->stream);
    if (h->rev) tempest_destroy(h->rev);
    h->rev = nullptr;
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    for (cudaEvent_t &e : h->kev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t &e : h->eev)
        if (e) cudaEventDestroy(e);
    free_all(h);
    if (h->hstat) cudaFreeHost(h->hstat);
    if (h->hpin) cudaFreeHost(h->hpin);
    delete h;
    return TEMPEST_OK;
}

int tempest_set_stream(tempest_t *h, void *stream)
{
    if (!h) return TEMPEST_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return TEMPEST_OK;
}

int tempest_set_allocator(tempest_t *h, void *(*alloc)(size_t, void *), void (*rel)(void *, void *), void *ctx,
                          size_t hbm_budget)
{
    if (!h) return TEMPEST_EINVAL;
    if (h->in_use > 0 && ((alloc != nullptr) != (h->alloc_fn != nullptr) || alloc != h->alloc_fn))
        return fail(h, TEMPEST_EINVAL, "tempest_set_allocator: must be called before the first allocation");
    if ((alloc == nullptr) != (rel == nullptr))
        return fail(h, TEMPEST_EINVAL, "tempest_set_allocator: alloc and release must both be set or both NULL");
    h->alloc_fn = alloc;
    h->release_fn = rel;
    h->alloc_ctx = ctx;
    h->budget = hbm_budget;
    return TEMPEST_OK;
}

int tempest_set_bias_params(tempest_t *h, double lambda_hop, double lambda_start)
{
    if (!h) return TEMPEST_EINVAL;
    if (!(lambda_hop > 0.0) || !(lambda_start >= 0.0))
        return fail(h, TEMPEST_EINVAL, "tempest_set_bias_params: need lambda_hop > 0 and lambda_start >= 0");
    h->lam_hop = lambda_hop;
    h->lam_start = lambda_start;
    return TEMPEST_OK;
}

int tempest_set_scheduler(tempest_t *h, int mode)
{
    if (!h) return TEMPEST_EINVAL;
    if (mode != TEMPEST_SCHED_FULL_WALK && mode != TEMPEST_SCHED_COOP && mode != TEMPEST_SCHED_STREAM &&
        mode != TEMPEST_SCHED_GRAPH && mode != TEMPEST_SCHED_LANE)
        return fail(h, TEMPEST_EINVAL, "tempest_set_scheduler: unknown mode %d", mode);
    h->sched = mode;
    return TEMPEST_OK;
}

int tempest_ingest(tempest_t *h, const int32_t *src, const int32_t *dst, const int64_t *ts, int64_t n,
                   tempest_ingest_stats *stats)
{
    if (!h) return TEMPEST_EINVAL;
    IngestUndo undo;
    int rc = ingest_batch(h, src, dst, ts, n, stats, &undo);
    if (rc || !h->rev) return rc;
    // the reversed index takes the same batch with the endpoints swapped; it
    // sees the same timestamps in the same order, so its window evicts the
    // same edges and its store stays position-aligned with the main one
    h->rev->stream = h->stream;
    rc = ingest_batch(h->rev, dst, src, ts, n, nullptr);
    if (rc) {
        // the in-edge index restored itself; the main index is undone too, so
        // that both hold the same edges and the call changed nothing
        const std::string why = h->rev->err;
        ingest_undo(h, undo);
        views_repair(h);  // best effort: a repair that fails is retried by the next call
        fail(h, rc, "tempest_ingest: the in-edge index failed (%s); the batch was not ingested", why.c_str());
    }
    return rc;
}

int tempest_enable_backward(tempest_t *h)
{
    if (!h) return TEMPEST_EINVAL;
    if (!h->directed || h->rev) return TEMPEST_OK;  // undirected graphs use their one view
    tempest_t *r = nullptr;
    int rc = tempest_create(h->window, 1, &r);
    if (rc) return fail(h, rc, "tempest_enable_backward: %s", tempest_last_error(nullptr));
    r->alloc_fn = h->alloc_fn;
    r->release_fn = h->release_fn;
    r->alloc_ctx = h->alloc_ctx;
    r->budget = h->budget;
    r->stream = h->stream;
    r->bkt_log = h->bkt_log;
    if (h->m > 0) {
        // the live edges, reversed, as one batch: they are in (ts, arrival)
        // order and inside the window, so the new index holds all of them in
        // the same order
        const int32_t *ss = h->st_src[h->cur].as<int32_t>() + h->s_lo;
        const int32_t *sd = h->st_dst[h->cur].as<int32_t>() + h->s_lo;
        const int64_t *st = h->st_ts[h->cur].as<int64_t>() + h->s_lo;
        rc = ingest_batch(r, sd, ss, st, h->m, nullptr);
        if (!rc && r->m != h->m) rc = fail(r, TEMPEST_ECUDA, "replay kept %lld of %lld edges", (long long)r->m,
                                           (long long)h->m);
        if (rc) {
            fail(h, rc, "tempest_enable_backward: %s", r->err.c_str());
            cudaStreamSynchronize(h->stream);
            tempest_destroy(r);
            return rc;
        }
    }
    // later batches meet the same late-arrival cutoff as the main index
    r->has_cutoff = h->has_cutoff;
    r->cutoff = h->cutoff;
    h->rev = r;
    return TEMPEST_OK;
}

static int active_nodes_dir(tempest_t *h, int direction, int64_t *n)
{
    if (!h || !n) return TEMPEST_EINVAL;
    tempest_t *vh = view_handle(h, direction);
    if (!vh) return fail(h, TEMPEST_EINVAL, "backward walks of a directed graph need tempest_enable_backward");
    int rc;
    if ((rc = prepare_active_nodes(vh))) return vh == h ? rc : fail(h, rc, "%s", vh->err.c_str());
    *n = vh->n_pn;
    return TEMPEST_OK;
}

int tempest_active_nodes(tempest_t *h, int64_t *n) { return active_nodes_dir(h, 0, n); }

int tempest_active_nodes_backward(tempest_t *h, int64_t *n) { return active_nodes_dir(h, 1, n); }

// Walk rows into host buffers.  The host link and the host's own stores move
// a few hundred GB/s each, and padding is most of a row, so the rows are
// split: a share of them (h->host_link_pct percent, a tuning knob) is padded
// on the device and copied whole, while for the rest only each walk's cells
// travel (gathered back to back on the device, with the lengths and offsets)
// and host threads write those rows and their padding, during the copy of the
// first part.  The first part is a band that either side may take: a copy
// thread hands it to the copy engine a chunk at a time from its bottom, two
// chunks ahead of the engine, and host threads that have written their own
// rows take it from the top (its cells travel with the host part's), so a
// copy that slows down (the link is shared with the host's other traffic)
// leaves less of the call undone.

static int walks_to_host(tempest_t *h, int64_t n, int32_t cap, int32_t *d_node, int64_t *d_ts, const int32_t *d_len,
                         int32_t *node, int64_t *ts, int32_t *len, bool dev_len)
{
    cudaStream_t st = h->stream;
    int rc;
    const int64_t nd = std::min<int64_t>(n, n * h->host_link_pct / 100);  // rows padded on the device
    const int64_t nb = (nd > 0 && nd < n) ? 0 : nd;  // rows [nb, nd): the band either side takes
    const int64_t nh = n - nb;                            // rows whose cells travel
    const size_t rowb = sizeof(int32_t) * (size_t)cap, rowt = sizeof(int64_t) * (size_t)cap;
    int64_t grid = (n + 255) / 256;
    const int64_t gcap = (int64_t)h->num_sms * 16;
    if (grid > gcap) grid = gcap;
    if (nd > 0) pad_rows(h, nd, cap, d_len, d_node, d_ts);
    if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
    if ((rc = ensure(h, h->cmp_off, sizeof(int64_t) * (size_t)(nh > 0 ? nh : 1) + 256, true))) return rc;
    int64_t *d_off = h->cmp_off.as<int64_t>();
    uint64_t *part = h->partials.as<uint64_t>();
    const int32_t *hlen_d = d_len + nb;
    const int nblk = scan_launch(LenScanOp{hlen_d, cap, d_off}, nh, part, st);
    uint64_t *hp = static_cast<uint64_t *>(h->hstat);
    cudaMemcpyAsync(hp, part + nblk, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "walks (compact)"))) return rc;
    const int64_t tot = nh > 0 ? (int64_t)hp[0] : 0;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_off = up(sizeof(int64_t) * (size_t)nh), b_node = up(sizeof(int32_t) * (size_t)tot),
                 b_ts = up(sizeof(int64_t) * (size_t)tot), b_len = up(sizeof(int32_t) * (size_t)n);
    if ((rc = ensure(h, h->cmp_stage, b_node + b_ts + 256, true))) return rc;
    int32_t *c_node = h->cmp_stage.as<int32_t>();
    int64_t *c_ts = reinterpret_cast<int64_t *>(h->cmp_stage.as<char>() + b_node);
    if (tot > 0)
        k_compact_rows<<<(unsigned)grid, 256, 0, st>>>(d_node + nb * (int64_t)cap, d_ts + nb * (int64_t)cap, hlen_d,
                                                       d_off, nh, cap, c_node, c_ts);
    if ((rc = ensure_pinned(h, b_off + b_node + b_ts + b_len + 256))) return rc;
    char *hb = static_cast<char *>(h->hpin);
    int64_t *h_off = reinterpret_cast<int64_t *>(hb);
    int32_t *h_node = reinterpret_cast<int32_t *>(hb + b_off);
    int64_t *h_ts = reinterpret_cast<int64_t *>(hb + b_off + b_node);
    int32_t *h_len = dev_len ? reinterpret_cast<int32_t *>(hb + b_off + b_node + b_ts) : len;
    // the host part's inputs first, then the whole rows
    cudaMemcpyAsync(h_len, d_len, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (nh > 0) cudaMemcpyAsync(h_off, d_off, sizeof(int64_t) * (size_t)nh, cudaMemcpyDeviceToHost, st);
    if (tot > 0) {
        cudaMemcpyAsync(h_node, c_node, sizeof(int32_t) * (size_t)tot, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(h_ts, c_ts, sizeof(int64_t) * (size_t)tot, cudaMemcpyDeviceToHost, st);
    }
    cudaEvent_t ev[4] = {};  // [0]: the host part's inputs are on the host; [1..3]: the copy thread's chunks
    for (cudaEvent_t &e : ev) {
        if ((rc = cuda_check(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "walks (host event)"))) {
            for (cudaEvent_t &x : ev)
                if (x) cudaEventDestroy(x);
            return rc;
        }
    }
    cudaEventRecord(ev[0], st);
    if (nb > 0) {
        cudaMemcpyAsync(node, d_node, rowb * (size_t)nb, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(ts, d_ts, rowt * (size_t)nb, cudaMemcpyDeviceToHost, st);
    }
    // the band: unclaimed rows [front, back), the copy thread's from the
    // bottom in chunks of copy_chunk rows, the host threads' from the top in
    // chunks of host_chunk rows
    std::mutex mu;
    int64_t front = nb, back = nd, band_copied = 0;
    int copy_err = 0;
    const int64_t band = nd - nb;
    const int64_t copy_chunk = std::min<int64_t>(65536, std::max<int64_t>(256, band / 16));
    const int64_t host_chunk = std::min<int64_t>(2048, std::max<int64_t>(64, band / 64));
    auto claim_bottom = [&](int64_t &a, int64_t &b) {
        std::lock_guard<std::mutex> g(mu);
        if (front >= back) return false;
        a = front;
        b = std::min(back, front + copy_chunk);
        front = b;
        return true;
    };
    auto claim_top = [&](int64_t &a, int64_t &b) {
        std::lock_guard<std::mutex> g(mu);
        if (back <= front) return false;
        b = back;
        a = std::max(front, back - host_chunk);
        back = a;
        return true;
    };
    // the copy thread keeps two chunks queued behind the engine's current
    // work, so that the rest of the band stays open to the host threads
    auto copier = [&]() {
        if (cudaSetDevice(h->device) != cudaSuccess) {
            cudaGetLastError();
            return;  // the host threads take the band
        }
        int64_t a, b;
        for (int64_t i = 0;; i++) {
            if (i >= 2 && cudaEventSynchronize(ev[1 + (i - 2) % 3]) != cudaSuccess) {
                copy_err = 1;
                break;
            }
            if (!claim_bottom(a, b)) break;
            cudaMemcpyAsync(node + a * (int64_t)cap, d_node + a * (int64_t)cap, rowb * (size_t)(b - a),
                            cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(ts + a * (int64_t)cap, d_ts + a * (int64_t)cap, rowt * (size_t)(b - a),
                            cudaMemcpyDeviceToHost, st);
            cudaEventRecord(ev[1 + i % 3], st);
            band_copied += b - a;
        }
    };
    std::thread cp;
    if (band > 0) {
        try {
            cp = std::thread(copier);
        } catch (...) {
            // no copy thread: the host threads take the whole band
        }
    }
    auto stop_copier = [&]() {
        {
            std::lock_guard<std::mutex> g(mu);
            back = front;
        }
        if (cp.joinable()) cp.join();
    };
    rc = cuda_check(h, cudaEventSynchronize(ev[0]), "walks (host outputs)");
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point a) { return std::chrono::duration<double, std::milli>(clk::now() - a).count(); };
    h->last_ws.host_ms[0] = ms_since(h->walk_t0);
    const clk::time_point t1 = clk::now();
    if (!rc) {
        // rows [nd, n), then rows of the band from its top, in parallel
        // threads (this one included) that take chunks of rows until none is
        // left: a thread that the host deschedules (its CPUs are shared)
        // delays one chunk, not a fixed share of the rows; a thread that
        // cannot start (no exception crosses the C ABI) leaves its chunks to
        // the others
        auto expand = [&](int64_t a, int64_t b) {
            expand_rows(a - nb, b - nb, cap, h_len + nb, h_off, h_node, h_ts, node + nb * (int64_t)cap,
                        ts + nb * (int64_t)cap);
        };
        constexpr int64_t CHUNK = 2048;
        std::atomic<int64_t> next{nd};
        auto work = [&]() {
            for (;;) {
                const int64_t i0 = next.fetch_add(CHUNK, std::memory_order_relaxed);
                if (i0 >= n) break;
                expand(i0, std::min(n, i0 + CHUNK));
            }
            int64_t a, b;
            while (claim_top(a, b)) expand(a, b);
        };
        const int64_t want = h->host_threads > 0 ? h->host_threads : std::min(host_cpus(), 32);
        const int64_t nt = std::min<int64_t>(want, std::max<int64_t>(1, nh / 4096));
        std::vector<std::thread> th;
        try {
            th.reserve((size_t)nt);
        } catch (...) {
        }
        for (int64_t k = 1; k < nt; k++) {
            try {
                th.emplace_back(work);
            } catch (...) {
            }
        }
        work();
        for (auto &x : th) x.join();
    }
    h->last_ws.host_ms[1] = ms_since(t1);
    const clk::time_point t2 = clk::now();
    stop_copier();
    const int rc2 = cuda_check(h, cudaStreamSynchronize(st), "walks (host outputs)");
    for (cudaEvent_t &e : ev) cudaEventDestroy(e);
    h->last_ws.host_ms[2] = ms_since(t2);
    if (rc) return rc;
    if (rc2) return rc2;
    if (copy_err) return fail(h, TEMPEST_ECUDA, "walks (host outputs): the copy thread failed");
    h->last_d2h = (int64_t)(sizeof(int32_t) * (size_t)n + sizeof(int64_t) * (size_t)nh + 12 * (size_t)tot +
                            (rowb + rowt) * (size_t)(nb + band_copied));
    return TEMPEST_OK;
}

static int walks_common(tempest_t *h, int64_t n_walks, int32_t cap, int32_t max_len, const int32_t *len_arr,
                        int bias, const uint8_t *bias_arr, int start_policy, uint64_t seed, int32_t *node,
                        int64_t *ts, int32_t *len, int direction = 0)
{
    int rc;
    tempest_t *vh = view_handle(h, direction);
    if (!vh) return fail(h, TEMPEST_EINVAL, "backward walks of a directed graph need tempest_enable_backward");
    if (direction && !bias_arr && bias == TEMPEST_BIAS_EXP_WEIGHT)
        return fail(h, TEMPEST_EINVAL, "walks: the weight-based bias runs forward only");
    if (!bias_arr && bias == TEMPEST_BIAS_NODE2VEC && h->n2v_q != 1.0 && !h->pt_on)
        return fail(h, TEMPEST_EINVAL, "walks: the Node2Vec pair table was dropped; call tempest_set_node2vec");
    if (n_walks < 0) return fail(h, TEMPEST_EINVAL, "walks: n_walks < 0");
    if (cap < 2) return fail(h, TEMPEST_EINVAL, "walks: max_len must be >= 2");
    if (start_policy < TEMPEST_START_UNIFORM_EDGE || start_policy > TEMPEST_START_PER_NODE)
        return fail(h, TEMPEST_EINVAL, "walks: unknown start policy %d", start_policy);
    if (!bias_arr && (bias < 0 || bias > 4)) return fail(h, TEMPEST_EINVAL, "walks: unknown bias %d", bias);
    if (n_walks > 0 && (!node || !ts || !len)) return fail(h, TEMPEST_EINVAL, "walks: NULL output");
    if (n_walks > 0 && (int64_t)cap * n_walks / n_walks != (int64_t)cap)
        return fail(h, TEMPEST_EINVAL, "walks: output size overflows");
    int64_t pn_k = 0;
    if ((rc = per_node_k(vh, start_policy, n_walks, pn_k, "walks")))
        return vh == h ? rc : fail(h, rc, "%s", vh->err.c_str());
    cudaStream_t st = h->stream;
    h->last_ws = tempest_walk_stats{};
    h->walk_t0 = std::chrono::steady_clock::now();
    if (n_walks == 0) return TEMPEST_OK;

    // per-walk inputs: validate on the host when they are host arrays
    const int32_t *d_len = len_arr;
    const uint8_t *d_bias = bias_arr;
    const bool host_len = len_arr && !is_device_ptr(len_arr);
    const bool host_bias = bias_arr && !is_device_ptr(bias_arr);
    if (host_len)
        for (int64_t i = 0; i < n_walks; i++)
            if (len_arr[i] < 2 || len_arr[i] > cap)
                return fail(h, TEMPEST_EINVAL, "walks_mixed: max_len_arr[%lld] = %d outside [2, %d]", (long long)i,
                            len_arr[i], cap);
    if (host_bias)
        for (int64_t i = 0; i < n_walks; i++)
            if (bias_arr[i] > 4 || (direction && bias_arr[i] == TEMPEST_BIAS_EXP_WEIGHT))
                return fail(h, TEMPEST_EINVAL, "walks_mixed: bias_arr[%lld] = %d unknown%s", (long long)i,
                            bias_arr[i], direction ? " for backward walks" : "");
    if (host_len || host_bias) {
        size_t need = 0;
        if (host_len) need += sizeof(int32_t) * (size_t)n_walks;
        if (host_bias) need += (size_t)n_walks + 16;
        if ((rc = ensure(h, h->in_stage, need, true))) return rc;
        char *p = h->in_stage.as<char>();
        if (host_len) {
            cudaMemcpyAsync(p, len_arr, sizeof(int32_t) * (size_t)n_walks, cudaMemcpyHostToDevice, st);
            d_len = reinterpret_cast<const int32_t *>(p);
            p += sizeof(int32_t) * (size_t)n_walks;
        }
        if (host_bias) {
            cudaMemcpyAsync(p, bias_arr, (size_t)n_walks, cudaMemcpyHostToDevice, st);
            d_bias = reinterpret_cast<const uint8_t *>(p);
        }
    }

    const bool dev_node = is_device_ptr(node), dev_ts = is_device_ptr(ts), dev_len = is_device_ptr(len);
    const size_t cells = (size_t)cap * (size_t)n_walks;
    int32_t *d_node = node;
    int64_t *d_ts = ts;
    int32_t *d_lenout = len;
    if (!dev_node || !dev_ts || !dev_len) {
        size_t need = 0;
        if (!dev_ts) need += sizeof(int64_t) * cells;
        if (!dev_node) need += sizeof(int32_t) * cells;
        if (!dev_len) need += sizeof(int32_t) * (size_t)n_walks;
        if ((rc = ensure(h, h->out_stage, need + 64, true))) return rc;
        char *p = h->out_stage.as<char>();
        if (!dev_ts) {
            d_ts = reinterpret_cast<int64_t *>(p);
            p += sizeof(int64_t) * cells;
        }
        if (!dev_node) {
            d_node = reinterpret_cast<int32_t *>(p);
            p += sizeof(int32_t) * cells;
        }
        if (!dev_len) d_lenout = reinterpret_cast<int32_t *>(p);
    }
    WalkRequest rq{n_walks, cap, max_len, d_len, bias, d_bias, start_policy, pn_k, seed, d_node, d_ts, d_lenout};
    rq.direction = direction;
    // host rows: the device keeps only each walk's cells, the host pads
    const bool compact = !dev_node && !dev_ts;
    rq.no_pad = compact ? 1 : 0;
    if (host_bias) {
        for (int64_t i = 0; i < n_walks && !rq.want_w; i++) rq.want_w = bias_arr[i] == TEMPEST_BIAS_EXP_WEIGHT;
        rq.may_n2v = 0;
        for (int64_t i = 0; i < n_walks && !rq.may_n2v; i++) rq.may_n2v = bias_arr[i] == TEMPEST_BIAS_NODE2VEC;
    }
    if ((rc = walks_run(h, rq))) return rc;
    h->last_d2h = 0;
    if (compact) return walks_to_host(h, n_walks, cap, d_node, d_ts, d_lenout, node, ts, len, dev_len);
    if (!dev_ts) cudaMemcpyAsync(ts, d_ts, sizeof(int64_t) * cells, cudaMemcpyDeviceToHost, st);
    if (!dev_node) cudaMemcpyAsync(node, d_node, sizeof(int32_t) * cells, cudaMemcpyDeviceToHost, st);
    if (!dev_len) cudaMemcpyAsync(len, d_lenout, sizeof(int32_t) * (size_t)n_walks, cudaMemcpyDeviceToHost, st);
    h->last_d2h = (int64_t)((dev_ts ? 0 : sizeof(int64_t) * cells) + (dev_node ? 0 : sizeof(int32_t) * cells) +
                            (dev_len ? 0 : sizeof(int32_t) * (size_t)n_walks));
    if (!dev_node || !dev_ts || !dev_len || host_len || host_bias)
        return cuda_check(h, cudaStreamSynchronize(st), "walks (host outputs)");
    return cuda_check(h, cudaGetLastError(), "walks");
}

int tempest_walks(tempest_t *h, int64_t n_walks, int32_t max_len, int bias, int start_policy, uint64_t seed,
                  int32_t *node, int64_t *ts, int32_t *len)
{
    if (!h) return TEMPEST_EINVAL;
    return walks_common(h, n_walks, max_len, max_len, nullptr, bias, nullptr, start_policy, seed, node, ts, len);
}

int tempest_walks_backward(tempest_t *h, int64_t n_walks, int32_t max_len, int bias, int start_policy,
                           uint64_t seed, int32_t *node, int64_t *ts, int32_t *len)
{
    if (!h) return TEMPEST_EINVAL;
    return walks_common(h, n_walks, max_len, max_len, nullptr, bias, nullptr, start_policy, seed, node, ts, len, 1);
}

int tempest_walks_mixed(tempest_t *h, int64_t n_walks, const int32_t *max_len_arr, int32_t max_len_cap,
                        const uint8_t *bias_arr, int start_policy, uint64_t seed, int32_t *node, int64_t *ts,
                        int32_t *len)
{
    if (!h) return TEMPEST_EINVAL;
    if (n_walks > 0 && (!max_len_arr || !bias_arr))
        return fail(h, TEMPEST_EINVAL, "tempest_walks_mixed: NULL max_len_arr or bias_arr");
    return walks_common(h, n_walks, max_len_cap, max_len_cap, max_len_arr, 0, bias_arr, start_policy, seed, node,
                        ts, len);
}

int tempest_sample_index(tempest_t *h, const uint64_t *u_bits, const int64_t *n, int64_t count, int bias,
                         double lambda, int64_t *out)
{
    if (!h) return TEMPEST_EINVAL;
    if (count < 0 || bias < 0 || bias > 2 || !(lambda > 0.0))
        return fail(h, TEMPEST_EINVAL, "tempest_sample_index: bad count, bias or lambda");
    if (count == 0) return TEMPEST_OK;
    if (!is_device_ptr(u_bits) || !is_device_ptr(n) || !is_device_ptr(out))
        return fail(h, TEMPEST_EINVAL, "tempest_sample_index: arrays must be device memory");
    return sample_index_run(h, u_bits, n, count, bias, lambda, out);
}

int tempest_last_walk_stats(tempest_t *h, tempest_walk_stats *out)
{
    if (!h || !out) return TEMPEST_EINVAL;
    int rc;
    if (h->wcnt.p) {
        WalkCounters *hc = static_cast<WalkCounters *>(h->hstat);
        cudaMemcpyAsync(hc, h->wcnt.p, sizeof(WalkCounters), cudaMemcpyDeviceToHost, h->stream);
        if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "walk stats"))) return rc;
        h->last_ws.hops = (int64_t)hc->hops;
        h->last_ws.model_bytes = (int64_t)hc->model_bytes;
        h->last_ws.d2h_bytes = h->last_d2h;
        if (h->kev_valid) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, h->kev[0], h->kev[1]) == cudaSuccess) h->last_ws.kernel_ms = ms;
        }
        if (hc->status) {
            *out = h->last_ws;
            return fail(h, TEMPEST_EINVAL, "walks_mixed: a per-walk max_len or bias was out of range "
                                           "(those walks were clamped)");
        }
    }
    *out = h->last_ws;
    return TEMPEST_OK;
}

int tempest_get_counts(tempest_t *h, int64_t out[10])
{
    if (!h || !out) return TEMPEST_EINVAL;
    out[0] = h->m;
    out[1] = h->G;
    out[2] = h->N;
    out[3] = h->M;
    out[4] = h->Gn;
    out[5] = h->dropped;
    out[6] = h->evicted;
    out[7] = h->has_cutoff;
    out[8] = h->cutoff;
    out[9] = h->seq_next;
    return TEMPEST_OK;
}

int tempest_export_state(tempest_t *h, int which, void *dst, int64_t cap, int64_t *n)
{
    if (!h) return TEMPEST_EINVAL;
    int64_t cnt;
    size_t esz;
    switch (which) {
        case TEMPEST_STATE_SRC: cnt = h->m; esz = 4; break;
        case TEMPEST_STATE_DST: cnt = h->m; esz = 4; break;
        case TEMPEST_STATE_TS: cnt = h->m; esz = 8; break;
        case TEMPEST_STATE_TS_GROUP_OFF: cnt = h->G + 1; esz = 4; break;
        case TEMPEST_STATE_NODE_OFF: cnt = h->N + 1; esz = 4; break;
        case TEMPEST_STATE_NODE_ORDER: cnt = h->M; esz = 4; break;
        case TEMPEST_STATE_NODE_GROUP_OFF: cnt = h->Gn + 1; esz = 4; break;
        case TEMPEST_STATE_NODE_GIDX: cnt = h->N + 1; esz = 4; break;
        default: return fail(h, TEMPEST_EINVAL, "tempest_export_state: unknown array %d", which);
    }
    if (n) *n = cnt;
    if (!dst) return TEMPEST_OK;
    if (cap < cnt) return fail(h, TEMPEST_EINVAL, "tempest_export_state: capacity %lld < %lld", (long long)cap,
                               (long long)cnt);
    if (cnt == 0) return TEMPEST_OK;
    cudaStream_t st = h->stream;
    const size_t bytes = esz * (size_t)cnt;
    const bool dev = is_device_ptr(dst);
    int rc;
    if ((rc = views_repair(h))) return rc;
    if (!h->nv_ready || !h->tg.p) {
        // nothing ingested yet: every remaining array is the single offset 0
        if (dev) return cuda_check(h, cudaMemsetAsync(dst, 0, bytes, st), "export");
        memset(dst, 0, bytes);
        return TEMPEST_OK;
    }
    const void *srcp = nullptr;
    switch (which) {
        case TEMPEST_STATE_SRC: srcp = h->st_src[h->cur].as<int32_t>() + h->s_lo; break;
        case TEMPEST_STATE_DST: srcp = h->st_dst[h->cur].as<int32_t>() + h->s_lo; break;
        case TEMPEST_STATE_TS: srcp = h->st_ts[h->cur].as<int64_t>() + h->s_lo; break;
        default: {
            // derived arrays are written to device memory first
            void *target = dst;
            if (!dev) {
                if ((rc = ensure(h, h->exp_stage, bytes))) return rc;
                target = h->exp_stage.p;
            }
            rc = which == TEMPEST_STATE_TS_GROUP_OFF ? ts_export(h, static_cast<int32_t *>(target))
                                                     : nv_export(h, which, static_cast<int32_t *>(target));
            if (rc) return rc;
            if (dev) return cuda_check(h, cudaStreamSynchronize(st), "export");
            srcp = target;
        }
    }
    cudaMemcpyAsync(dst, srcp, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    return cuda_check(h, cudaStreamSynchronize(st), "export");
}

int tempest_sync(tempest_t *h)
{
    if (!h) return TEMPEST_EINVAL;
    return cuda_check(h, cudaStreamSynchronize(h->stream), "tempest_sync");
}

}  // extern "C"
