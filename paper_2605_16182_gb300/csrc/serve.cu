// serve.cu -- batched walk requests and the serving loop.
//
// tempest_walks_batch runs several walk requests in one persistent launch.
// The server keeps a FIFO of ingest and walk requests over the device-
// resident index and advances it without blocking:
//   * walk requests are admitted in arrival order into a wave while the wave
//     has launch slots (max_wave_walks) and their outputs fit in an output
//     arena of a fixed HBM budget; a wave is one multi-request launch;
//   * up to two waves are in flight on two streams, so requests that arrive
//     while a wave runs start in the next wave and overlap its tail;
//   * an ingest request waits until no wave is in flight (every earlier walk
//     request sees the index state of its arrival), then runs;
//   * a completed request's arena memory returns when the client releases it.
// A walk draws from Philox(seed, walk, hop) of its own request, so a request
// gives the same walks alone or in any mix.
#include <chrono>
#include <new>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

#include "engine.cuh"
#include "walkcore.cuh"

namespace tw {

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Validates requests and lays out their descriptors with offsets.
static int build_table(tempest_t *h, const tempest_walk_request *reqs, int n, ReqDesc *out, int64_t &total)
{
    total = 0;
    for (int i = 0; i < n; i++) {
        const tempest_walk_request &q = reqs[i];
        if (q.n_walks < 0 || q.max_len < 2 || q.start_policy < 0 || q.start_policy > TEMPEST_START_PER_NODE ||
            (!q.bias_arr && (q.bias < 0 || q.bias > 4)))
            return fail(h, TEMPEST_EINVAL, "walk request %d: bad n_walks, max_len, bias or start policy", i);
        if (q.n_walks > 0 && (!is_device_ptr(q.node) || !is_device_ptr(q.ts) || !is_device_ptr(q.len)))
            return fail(h, TEMPEST_EINVAL, "walk request %d: outputs must be device memory", i);
        if ((q.max_len_arr && !is_device_ptr(q.max_len_arr)) || (q.bias_arr && !is_device_ptr(q.bias_arr)))
            return fail(h, TEMPEST_EINVAL, "walk request %d: per-walk arrays must be device memory", i);
        if (q.direction != 0 && q.direction != 1)
            return fail(h, TEMPEST_EINVAL, "walk request %d: direction %d is neither 0 nor 1", i, q.direction);
        if (q.direction == 1 && !q.bias_arr && q.bias == TEMPEST_BIAS_EXP_WEIGHT)
            return fail(h, TEMPEST_EINVAL, "walk request %d: backward walks take biases 0-2", i);
        tempest_t *vh = view_handle(h, q.direction);
        if (!vh)
            return fail(h, TEMPEST_EINVAL, "walk request %d: backward walks of a directed graph need "
                        "tempest_enable_backward", i);
        ReqDesc &d = out[i];
        int rc = per_node_k(vh, q.start_policy, q.n_walks, d.pn_k, "walk request");
        if (rc && vh != h) fail(h, rc, "%s", vh->err.c_str());
        if (rc) return rc;
        d.n_walks = q.n_walks;
        d.offset = total;
        d.len_arr = q.max_len_arr;
        d.bias_arr = q.bias_arr;
        d.node = q.node;
        d.ts = q.ts;
        d.len = q.len;
        d.seed = q.seed;
        d.cap = q.max_len;
        d.max_len = q.max_len;
        d.bias = q.bias;
        d.start_policy = q.start_policy;
        total += q.n_walks;
    }
    return TEMPEST_OK;
}

// Derived indexes of a launch in the given direction: the time-bucket tables
// of the view it reads, and (forward) the weight sums when a request asks for
// the weight-based bias, or may (device per-walk biases) once weights are kept.
static int prepare_for(tempest_t *h, int direction, const ReqDesc *t, int n)
{
    tempest_t *vh = view_handle(h, direction);
    if (!vh) return fail(h, TEMPEST_EINVAL, "backward walks of a directed graph need tempest_enable_backward");
    int rc = prepare_walk_index(vh);
    if (rc) {
        if (vh != h) fail(h, rc, "%s", vh->err.c_str());
        return rc;
    }
    if (direction) return TEMPEST_OK;
    for (int i = 0; i < n; i++)
        if ((!t[i].bias_arr && t[i].bias == TEMPEST_BIAS_EXP_WEIGHT) || (t[i].bias_arr && h->w_on))
            return prepare_weights(h);
    return TEMPEST_OK;
}

// Whether a launch table may hold Node2Vec walks (a per-walk bias array, or
// that scalar bias).
static bool table_may_n2v(const ReqDesc *t, int n)
{
    for (int i = 0; i < n; i++)
        if (t[i].bias_arr || t[i].bias == TEMPEST_BIAS_NODE2VEC) return true;
    return false;
}

// Requests with no walks are dropped from a launch table (offsets stay
// consistent: they occupy no walk ids).
static int compact_table(ReqDesc *t, int n)
{
    int k = 0;
    for (int i = 0; i < n; i++)
        if (t[i].n_walks > 0) t[k++] = t[i];
    return k;
}

}  // namespace tw

using namespace tw;

struct tempest_server {
    tempest_t *h = nullptr;
    size_t arena_bytes = 0;
    DBuf arena;
    std::map<size_t, size_t> free_blocks;  // offset -> size
    int64_t max_wave_walks = 0;
    int max_inflight = 2;
    struct Req {
        int kind = 0;  // 0 walks, 1 ingest
        tempest_walk_request w{};
        const int32_t *src = nullptr, *dst = nullptr;
        const int64_t *ts = nullptr;
        int64_t n = 0;
        int state = 0;  // 0 queued, 1 running, 2 done, < 0 failed
        bool arena_out = false;
        size_t off = 0, bytes = 0;
        double t_submit = 0, t_start = 0, t_done = 0;
    };
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<uint64_t> queue;
    uint64_t next_id = 1;
    struct Wave {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        DBuf table;                // ReqDesc[max] + WalkCounters
        ReqDesc *stage = nullptr;  // pinned host staging
        int cap = 0;
        std::vector<uint64_t> ids;
        bool busy = false;
    };
    Wave waves[2];
    cudaEvent_t order_ev = nullptr;  // orders waves after the handle's stream
    int64_t n_waves = 0, n_ingests = 0, n_wave_requests = 0;
};

namespace {

bool arena_alloc(tempest_server *s, size_t bytes, size_t &off)
{
    for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
        if (it->second >= bytes) {
            off = it->first;
            const size_t rest = it->second - bytes;
            s->free_blocks.erase(it);
            if (rest) s->free_blocks[off + bytes] = rest;
            return true;
        }
    }
    return false;
}

void arena_free(tempest_server *s, size_t off, size_t bytes)
{
    auto it = s->free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_blocks.erase(nx);
    }
    if (it != s->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_blocks.erase(it);
        }
    }
}

size_t out_bytes(const tempest_walk_request &w)
{
    const size_t cells = (size_t)w.n_walks * (size_t)w.max_len;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return up(cells * 8) + up(cells * 4) + up((size_t)w.n_walks * 4);
}

int ensure_wave_table(tempest_server *s, tempest_server::Wave &wv, int n)
{
    if (wv.cap >= n) return TEMPEST_OK;
    int cap = wv.cap ? wv.cap : 64;
    while (cap < n) cap *= 2;
    const size_t bytes = sizeof(ReqDesc) * (size_t)cap + sizeof(WalkCounters) + 256;
    int rc = ensure(s->h, wv.table, bytes);
    if (rc) return rc;
    if (wv.stage) cudaFreeHost(wv.stage);
    wv.stage = nullptr;
    if (cudaMallocHost((void **)&wv.stage, sizeof(ReqDesc) * (size_t)cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(s->h, TEMPEST_ENOMEM, "server: pinned staging");
    }
    wv.cap = cap;
    return TEMPEST_OK;
}

// Launches one wave from the head of the queue; returns the number of
// requests it took (0 when the head cannot be admitted yet).
int launch_wave(tempest_server *s, tempest_server::Wave &wv, int &rc)
{
    rc = TEMPEST_OK;
    std::vector<uint64_t> ids;
    std::vector<tempest_walk_request> wr;
    int64_t walks = 0;
    while (!s->queue.empty()) {
        const uint64_t id = s->queue.front();
        tempest_server::Req &r = s->reqs[id];
        if (r.kind != 0) break;
        if (!ids.empty() && walks + r.w.n_walks > s->max_wave_walks) break;
        if (!ids.empty() && r.w.direction != wr[0].direction) break;  // a wave reads one view
        if (r.arena_out && r.bytes == 0) {
            const size_t b = out_bytes(r.w);
            if (b > s->arena_bytes) {  // can never fit
                r.state = TEMPEST_ENOMEM;
                r.t_done = now_s();
                s->queue.pop_front();
                continue;
            }
            size_t off;
            if (!arena_alloc(s, b, off)) break;  // wait for memory (FIFO)
            r.off = off;
            r.bytes = b;
            char *base = s->arena.as<char>() + off;
            const size_t cells = (size_t)r.w.n_walks * (size_t)r.w.max_len;
            auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
            r.w.ts = reinterpret_cast<int64_t *>(base);
            r.w.node = reinterpret_cast<int32_t *>(base + up(cells * 8));
            r.w.len = reinterpret_cast<int32_t *>(base + up(cells * 8) + up(cells * 4));
        }
        ids.push_back(id);
        wr.push_back(r.w);
        walks += r.w.n_walks;
        s->queue.pop_front();
    }
    if (ids.empty()) return 0;
    if ((rc = ensure_wave_table(s, wv, (int)ids.size()))) return 0;
    int64_t total = 0;
    if ((rc = build_table(s->h, wr.data(), (int)wr.size(), wv.stage, total))) {
        for (uint64_t id : ids) {
            s->reqs[id].state = rc;
            s->reqs[id].t_done = now_s();
        }
        return (int)ids.size();
    }
    const int n = compact_table(wv.stage, (int)ids.size());
    // derived walk indexes of the current state, built on the handle's stream
    const int dir = wr[0].direction;
    if ((rc = prepare_for(s->h, dir, wv.stage, n))) {
        for (uint64_t id : ids) {
            s->reqs[id].state = rc;
            s->reqs[id].t_done = now_s();
        }
        return (int)ids.size();
    }
    // the wave runs after everything queued on the handle's stream so far
    // (for example the kernels that produced or last used its buffers)
    cudaEventRecord(s->order_ev, s->h->stream);
    cudaStreamWaitEvent(wv.st, s->order_ev, 0);
    ReqDesc *dtab = wv.table.as<ReqDesc>();
    WalkCounters *cnt = reinterpret_cast<WalkCounters *>(wv.table.as<char>() + sizeof(ReqDesc) * (size_t)wv.cap);
    cudaMemcpyAsync(dtab, wv.stage, sizeof(ReqDesc) * (size_t)(n > 0 ? n : 1), cudaMemcpyHostToDevice, wv.st);
    rc = walks_multi_launch(s->h, dir, dtab, n, total, cnt, wv.st, true, table_may_n2v(wv.stage, n));
    cudaEventRecord(wv.ev, wv.st);
    const double t = now_s();
    for (uint64_t id : ids) {
        s->reqs[id].state = 1;
        s->reqs[id].t_start = t;
    }
    wv.ids = ids;
    wv.busy = true;
    s->n_waves++;
    s->n_wave_requests += (int64_t)ids.size();
    return (int)ids.size();
}

}  // namespace

// A host allocation inside a C ABI call failed (the containers of the
// request queue and the wave tables): report it as ENOMEM.
static int host_oom(tempest_t *h, const char *what) noexcept
{
    try {
        if (h) fail(h, TEMPEST_ENOMEM, "%s: host memory exhausted", what);
    } catch (...) {
    }
    return TEMPEST_ENOMEM;
}

extern "C" {

int tempest_walks_batch(tempest_t *h, const tempest_walk_request *reqs, int n_req)
{
    try {
        if (!h) return TEMPEST_EINVAL;
        if (n_req < 0 || (n_req > 0 && !reqs)) return fail(h, TEMPEST_EINVAL, "tempest_walks_batch: bad request list");
        h->last_ws = tempest_walk_stats{};
        if (n_req == 0) return TEMPEST_OK;
        // one launch per direction present (a launch reads one view); each
        // direction's requests keep their own offsets from 0
        std::vector<tempest_walk_request> part[2];
        for (int i = 0; i < n_req; i++) part[reqs[i].direction == 1 ? 1 : 0].push_back(reqs[i]);
        std::vector<ReqDesc> tab[2];
        int64_t total[2] = {0, 0};
        int n[2] = {0, 0};
        int rc;
        for (int d = 0; d < 2; d++) {
            // validation runs on the caller's request list order within a direction
            tab[d].resize(part[d].size());
            if (part[d].empty()) continue;
            if ((rc = build_table(h, part[d].data(), (int)part[d].size(), tab[d].data(), total[d]))) return rc;
            n[d] = compact_table(tab[d].data(), (int)part[d].size());
        }
        const size_t tb0 = (sizeof(ReqDesc) * (size_t)(n[0] > 0 ? n[0] : 1) + 255) & ~(size_t)255;
        const size_t tb1 = sizeof(ReqDesc) * (size_t)(n[1] > 0 ? n[1] : 1);
        if ((rc = ensure(h, h->in_stage, tb0 + tb1 + 256, true))) return rc;
        if ((rc = ensure(h, h->wcnt, sizeof(WalkCounters)))) return rc;
        char *stage = h->in_stage.as<char>();
        // the tables are small: a synchronous copy keeps the host arrays reusable
        for (int d = 0; d < 2; d++)
            if (n[d] && (rc = cuda_check(h, cudaMemcpyAsync(stage + (d ? tb0 : 0), tab[d].data(), sizeof(ReqDesc) * n[d],
                                                            cudaMemcpyHostToDevice, h->stream),
                                         "batch table")))
                return rc;
        if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "batch table"))) return rc;
        h->kev_valid = false;
        int launches = 0;
        for (int d = 0; d < 2; d++) {
            if (!n[d] && (d == 1 || n[1])) continue;  // an empty batch still clears the counters
            if ((rc = prepare_for(h, d, tab[d].data(), n[d]))) return rc;
            // the second launch adds to the first one's counters
            rc = walks_multi_launch(h, d, reinterpret_cast<ReqDesc *>(stage + (d ? tb0 : 0)), n[d], total[d],
                                    h->wcnt.as<WalkCounters>(), h->stream, launches == 0,
                                    table_may_n2v(tab[d].data(), n[d]));
            if (rc) return rc;
            launches++;
        }
        h->last_ws.n_walks = total[0] + total[1];
        h->last_ws.launches = launches;
        return cuda_check(h, cudaGetLastError(), "walks batch");
    } catch (...) {  // no C++ exception crosses the C ABI
        return host_oom(h, "tempest_walks_batch");
    }
}

int tempest_server_create(tempest_t *h, size_t arena_bytes, int64_t max_wave_walks, int max_inflight,
                          tempest_server **out)
{
    if (!h || !out || max_wave_walks <= 0 || max_inflight < 1 || max_inflight > 2)
        return fail(h, TEMPEST_EINVAL, "tempest_server_create: bad arguments");
    *out = nullptr;
    tempest_server *s = new (std::nothrow) tempest_server();
    if (!s) return fail(h, TEMPEST_ENOMEM, "tempest_server_create: host memory");
    s->h = h;
    s->arena_bytes = arena_bytes;
    s->max_wave_walks = max_wave_walks;
    s->max_inflight = max_inflight;
    int rc = TEMPEST_OK;
    if (arena_bytes) {
        rc = ensure(h, s->arena, arena_bytes);
        if (!rc) s->free_blocks[0] = arena_bytes;
    }
    if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&s->order_ev, cudaEventDisableTiming), "server event");
    for (int i = 0; i < 2 && !rc; i++) {
        rc = cuda_check(h, cudaStreamCreateWithFlags(&s->waves[i].st, cudaStreamNonBlocking), "server stream");
        if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&s->waves[i].ev, cudaEventDisableTiming), "server event");
    }
    if (rc) {
        tempest_server_destroy(s);
        return rc;
    }
    *out = s;
    return TEMPEST_OK;
}

int tempest_server_destroy(tempest_server *s)
{
    if (!s) return TEMPEST_OK;
    for (auto &wv : s->waves) {
        if (wv.st) cudaStreamSynchronize(wv.st);
        if (wv.ev) cudaEventDestroy(wv.ev);
        if (wv.st) cudaStreamDestroy(wv.st);
        if (wv.stage) cudaFreeHost(wv.stage);
        release(s->h, wv.table);
    }
    release(s->h, s->arena);
    if (s->order_ev) cudaEventDestroy(s->order_ev);
    delete s;
    return TEMPEST_OK;
}

int tempest_server_submit_walks(tempest_server *s, const tempest_walk_request *req, uint64_t *ticket)
{
    try {
        if (!s || !req || !ticket) return TEMPEST_EINVAL;
        tempest_server::Req r;
        r.kind = 0;
        r.w = *req;
        r.arena_out = !req->node && !req->ts && !req->len;
        if (r.arena_out && !s->arena_bytes)
            return fail(s->h, TEMPEST_EINVAL, "server: request without outputs and no output arena");
        r.t_submit = now_s();
        const uint64_t id = s->next_id++;
        s->reqs.emplace(id, r);
        s->queue.push_back(id);
        *ticket = id;
        return TEMPEST_OK;
    } catch (...) {  // no C++ exception crosses the C ABI
        return host_oom(s ? s->h : nullptr, "tempest_server_submit_walks");
    }
}

int tempest_server_submit_ingest(tempest_server *s, const int32_t *src, const int32_t *dst, const int64_t *ts,
                                 int64_t n, uint64_t *ticket)
{
    try {
        if (!s || !ticket) return TEMPEST_EINVAL;
        tempest_server::Req r;
        r.kind = 1;
        r.src = src;
        r.dst = dst;
        r.ts = ts;
        r.n = n;
        r.t_submit = now_s();
        const uint64_t id = s->next_id++;
        s->reqs.emplace(id, r);
        s->queue.push_back(id);
        *ticket = id;
        return TEMPEST_OK;
    } catch (...) {  // no C++ exception crosses the C ABI
        return host_oom(s ? s->h : nullptr, "tempest_server_submit_ingest");
    }
}

int tempest_server_progress(tempest_server *s, int *n_completed)
{
    try {
        if (!s) return TEMPEST_EINVAL;
        int done = 0;
        for (auto &wv : s->waves) {
            if (!wv.busy) continue;
            const cudaError_t e = cudaEventQuery(wv.ev);
            if (e == cudaErrorNotReady) continue;
            int st = (e == cudaSuccess) ? 2 : TEMPEST_ECUDA;
            if (e != cudaSuccess) cudaGetLastError();
            if (st == 2) {
                WalkCounters hc;
                const WalkCounters *cnt =
                    reinterpret_cast<const WalkCounters *>(wv.table.as<char>() + sizeof(ReqDesc) * (size_t)wv.cap);
                if (cudaMemcpy(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost) != cudaSuccess) {
                    cudaGetLastError();
                    st = TEMPEST_ECUDA;
                } else if (hc.status) {
                    st = TEMPEST_EINVAL;  // a request table or per-walk check failed
                    fail(s->h, TEMPEST_EINVAL, "server: wave check failed (code 0x%llx)", (unsigned long long)hc.status);
                }
            }
            const double t = now_s();
            for (uint64_t id : wv.ids) {
                s->reqs[id].state = st;
                s->reqs[id].t_done = t;
                done++;
            }
            wv.ids.clear();
            wv.busy = false;
        }
        int rc = TEMPEST_OK;
        while (!s->queue.empty()) {
            const uint64_t id = s->queue.front();
            tempest_server::Req &r = s->reqs[id];
            if (r.kind == 1) {
                bool busy = false;
                for (auto &wv : s->waves) busy |= wv.busy;
                if (busy) break;  // ingest is an epoch barrier
                r.t_start = now_s();
                r.state = 1;
                const int irc = tempest_ingest(s->h, r.src, r.dst, r.ts, r.n, nullptr);
                r.state = irc ? irc : 2;
                r.t_done = now_s();
                s->queue.pop_front();
                s->n_ingests++;
                done++;
                continue;
            }
            int free_slot = -1, inflight = 0;
            for (int i = 0; i < 2; i++) {
                if (s->waves[i].busy) inflight++;
                else if (free_slot < 0) free_slot = i;
            }
            if (free_slot < 0 || inflight >= s->max_inflight) break;
            const int took = launch_wave(s, s->waves[free_slot], rc);
            if (rc) break;
            if (took == 0) break;  // head waits for output memory
        }
        if (n_completed) *n_completed = done;
        return rc;
    } catch (...) {  // no C++ exception crosses the C ABI
        return host_oom(s ? s->h : nullptr, "tempest_server_progress");
    }
}

int tempest_server_status(tempest_server *s, uint64_t ticket, int *state, int32_t **node, int64_t **ts,
                          int32_t **len, double *latency_s)
{
    if (!s) return TEMPEST_EINVAL;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(s->h, TEMPEST_EINVAL, "server: unknown ticket");
    const tempest_server::Req &r = it->second;
    if (state) *state = r.state;
    if (node) *node = r.w.node;
    if (ts) *ts = r.w.ts;
    if (len) *len = r.w.len;
    if (latency_s) *latency_s = r.state >= 2 || r.state < 0 ? r.t_done - r.t_submit : -1.0;
    return TEMPEST_OK;
}

int tempest_server_release(tempest_server *s, uint64_t ticket)
{
    if (!s) return TEMPEST_EINVAL;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(s->h, TEMPEST_EINVAL, "server: unknown ticket");
    if (it->second.state == 0 || it->second.state == 1)
        return fail(s->h, TEMPEST_EBUSY, "server: request %llu still queued or running", (unsigned long long)ticket);
    if (it->second.bytes) arena_free(s, it->second.off, it->second.bytes);
    s->reqs.erase(it);
    return TEMPEST_OK;
}

int tempest_server_drain(tempest_server *s)
{
    try {
        if (!s) return TEMPEST_EINVAL;
        int rc = TEMPEST_OK;
        while (true) {
            int n = 0;
            if ((rc = tempest_server_progress(s, &n))) return rc;
            bool busy = !s->queue.empty();
            for (auto &wv : s->waves) busy |= wv.busy;
            if (!busy) return TEMPEST_OK;
            bool waiting = false;
            for (auto &wv : s->waves)
                if (wv.busy) {
                    cudaEventSynchronize(wv.ev);
                    waiting = true;
                }
            if (!waiting && !s->queue.empty()) {
                // the head waits for arena memory that only a release can free
                return fail(s->h, TEMPEST_EBUSY, "server: queue head needs output memory held by unreleased results");
            }
        }
    } catch (...) {  // no C++ exception crosses the C ABI
        return host_oom(s ? s->h : nullptr, "tempest_server_drain");
    }
}

int tempest_server_stats(tempest_server *s, int64_t out[4])
{
    if (!s || !out) return TEMPEST_EINVAL;
    out[0] = s->n_waves;
    out[1] = s->n_wave_requests;
    out[2] = s->n_ingests;
    out[3] = (int64_t)s->queue.size();
    return TEMPEST_OK;
}

}  // extern "C"
