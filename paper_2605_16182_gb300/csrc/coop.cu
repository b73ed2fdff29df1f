// coop.cu -- hierarchical cooperative scheduling of walk hops (Tempest
// Sec. 2.4.3-2.4.5, Algorithm 1).
//
// After the start step every live walk sits at some node.  Each hop step:
//   1. sorts the active walks by current node (stable radix sort of
//      (node, walk) pairs) -- the per-step regrouping;
//   2. finds the runs of walks at the same node (W = run length) and reads the
//      node's group count G;
//   3. classifies each run: W <= w_warp -> solo (one thread per run's walks),
//      W <= block_dim -> warp tier, else block tier; inside the cooperative
//      tiers G <= cap -> the node's group timestamps are staged in shared
//      memory ("smem"), otherwise read from global memory ("global"); a block
//      task with W > mega_split is split into ceil(W / mega_split) sub-tasks;
//   4. reads the five task counts on the host (sync 1), launches the five
//      terminal kernels, and reads the number of walks still active (sync 2).
// A hop of walk w draws from Philox(seed, w, hop) exactly as the other walk
// forms do, so every form returns the same walks.
#include "engine.cuh"
#include "prims.cuh"
#include "sortscan.cuh"
#include "walkcore.cuh"

namespace tw {

namespace {

enum { T_SOLO = 0, T_WARP_SMEM, T_WARP_GLOBAL, T_BLOCK_SMEM, T_BLOCK_GLOBAL, T_COUNT };

constexpr int COOP_BLOCK = 256;                 // block tier threads; the warp / block boundary
constexpr int COOP_WARPS = COOP_BLOCK / 32;
constexpr int SMEM_BYTES = 48 * 1024;           // static smem budget of one block
constexpr int BLOCK_G_CAP = SMEM_BYTES / 8;     // group timestamps one block can stage
constexpr int WARP_G_CAP = BLOCK_G_CAP / COOP_WARPS;

struct Task {
    int32_t node;
    int32_t start;  // first position in the node-sorted walk list
    int32_t count;  // walks
    int32_t pad;
};

struct CoopState {
    int32_t *ws_node;   // current node of each walk
    int64_t *ws_t;      // current time
    int32_t *ws_len;    // nodes written so far
    int32_t *ws_prev;   // the node before the current one (Node2Vec; -1: none)
    const uint32_t *sorted_walks;
    int32_t *next_active;
    unsigned int *n_next;
};

struct ActiveKeyLoader {
    const int32_t *active;
    const int32_t *ws_node;
    __device__ __forceinline__ uint32_t key(int64_t i) const { return (uint32_t)ws_node[active[i]]; }
    __device__ __forceinline__ uint32_t val(int64_t i) const { return (uint32_t)active[i]; }
};

struct RunOp {
    const uint32_t *K;
    int32_t *run_pos;
    int32_t *run_node;
    __device__ __forceinline__ uint64_t value(int64_t i) const { return (i == 0 || K[i] != K[i - 1]) ? 1u : 0u; }
    __device__ __forceinline__ void emit(int64_t i, uint64_t v, uint64_t ex) const
    {
        if (v) {
            run_pos[ex] = (int32_t)i;
            run_node[ex] = (int32_t)K[i];
        }
    }
};

}  // namespace

// Start edges of all walks; walks that can go on join the active list.
__global__ void __launch_bounds__(256) k_coop_start(const WalkView V, const WalkOut O, CoopState S)
{
    unsigned long long hops = 0, bytes = 0;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < O.n_walks; base += stride) {
        const int64_t w = base + lane;
        if (w < O.n_walks) {
            int32_t L;
            int bias;
            walk_params(O, w, L, bias);
            int32_t *nrow = O.node + w * (int64_t)O.cap;
            int64_t *trow = O.ts + w * (int64_t)O.cap;
            if (V.m == 0) {
                O.len[w] = 0;
            } else {
                int32_t s = -1, d, len0;
                int64_t t0;
                if (O.start_policy == TEMPEST_START_PER_NODE) {
                    // the walk starts at an active node before every live edge
                    d = __ldg(V.pn_nodes + w / O.pn_k);
                    t0 = pernode_time(V);
                    nrow[0] = d;
                    trow[0] = INT64_MIN;
                    len0 = 1;
                } else {
                    start_edge(V, O, w, bias, s, d, t0);
                    nrow[0] = s;
                    nrow[1] = d;
                    trow[0] = INT64_MIN;
                    trow[1] = t0;
                    t0 = search_time(V, t0);
                    hops++;
                    bytes += START_MODEL_BYTES;
                    len0 = 2;
                }
                if (L <= len0) {
                    O.len[w] = len0;
                } else {
                    S.ws_node[w] = d;
                    S.ws_t[w] = t0;
                    S.ws_len[w] = len0;
                    S.ws_prev[w] = len0 == 2 ? s : -1;
                    const unsigned am = __activemask();
                    const int leader = __ffs(am) - 1;
                    unsigned slot = 0;
                    if (lane == leader) slot = atomicAdd(S.n_next, (unsigned)__popc(am));
                    slot = __shfl_sync(am, slot, leader);
                    S.next_active[slot + __popc(am & ((1u << lane) - 1u))] = (int32_t)w;
                }
            }
        }
    }
    hops = warp_sum(hops);
    bytes = warp_sum(bytes);
    if (lane == 0 && hops) {
        atomicAdd(&O.cnt->hops, hops);
        atomicAdd(&O.cnt->model_bytes, bytes);
    }
}

__global__ void k_coop_classify(const int32_t *__restrict__ run_pos, const int32_t *__restrict__ run_node,
                                const uint64_t *__restrict__ n_runs_ptr, int64_t n_active,
                                const NodeRange *__restrict__ ngr, int w_warp, int mega, Task *tasks,
                                int64_t tier_stride, unsigned int *counts)
{
    const int64_t R = (int64_t)*n_runs_ptr;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t start = run_pos[r];
        const int32_t end = (r + 1 < R) ? run_pos[r + 1] : (int32_t)n_active;
        const int32_t W = end - start;
        const int32_t v = run_node[r];
        const int32_t G = ngr[v].g_hi - ngr[v].g_lo;
        int tier;
        if (W <= w_warp) tier = T_SOLO;
        else if (W <= COOP_BLOCK) tier = (G <= WARP_G_CAP) ? T_WARP_SMEM : T_WARP_GLOBAL;
        else tier = (G <= BLOCK_G_CAP) ? T_BLOCK_SMEM : T_BLOCK_GLOBAL;
        if (tier == T_BLOCK_SMEM || tier == T_BLOCK_GLOBAL) {
            const int32_t parts = (W + mega - 1) / mega;  // mega-hub split
            const unsigned base = atomicAdd(&counts[tier], (unsigned)parts);
            for (int32_t p = 0; p < parts; p++) {
                const int32_t s0 = start + p * mega;
                tasks[tier * tier_stride + base + p] = Task{v, s0, min(mega, end - s0), 0};
            }
        } else {
            const unsigned base = atomicAdd(&counts[tier], 1u);
            tasks[tier * tier_stride + base] = Task{v, start, W, 0};
        }
    }
}

// One hop of walk w at node v whose groups are [g0, g1); gts_local (when not
// null) holds the node's group timestamps in shared memory.
__device__ __forceinline__ void coop_hop(const WalkView &V, const WalkOut &O, const CoopState &S, int32_t w,
                                         int32_t v, int32_t g0, int32_t g1, const int64_t *gts_local,
                                         unsigned long long &hops, unsigned long long &bytes, bool &push)
{
    push = false;
    int32_t L;
    int bias;
    walk_params(O, w, L, bias);
    const int64_t t = S.ws_t[w];
    int32_t len = S.ws_len[w];
    int32_t c;
    if (gts_local) {
        int32_t lo = 0, hi = g1 - g0;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (gts_local[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        c = g0 + lo;
    } else {
        c = first_later(V, v, g0, g1, t);
    }
    if (V.back ? c == g0 : c == g1) {
        O.len[w] = len;  // Gamma_t(v) is empty
        return;
    }
    Entry e;
    if (bias == BIAS_NODE2VEC) {
        if (!draw_n2v(V, O, w, (uint32_t)(len - 1), g0, c, g1, S.ws_prev[w], e, bytes)) {
            O.len[w] = len;  // every proposal rejected
            return;
        }
        S.ws_prev[w] = v;
    } else {
        e = V.back ? draw_entry_back(V, O, w, (uint32_t)(len - 1), bias, g0, c)
                   : draw_entry(V, O, w, (uint32_t)(len - 1), bias, c, g1);
    }
    O.node[w * (int64_t)O.cap + len] = e.other;
    O.ts[w * (int64_t)O.cap + len] = e.ts;
    hops++;
    bytes += hop_model_bytes((int64_t)(g1 - g0));
    len++;
    if (len >= L) {
        O.len[w] = len;
        return;
    }
    S.ws_node[w] = e.other;
    S.ws_t[w] = search_time(V, e.ts);
    S.ws_len[w] = len;
    push = true;
}

__device__ __forceinline__ void push_active(const CoopState &S, bool push, int32_t w)
{
    const unsigned am = __activemask();
    const unsigned pm = __ballot_sync(am, push);
    if (!pm) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(pm) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(S.n_next, (unsigned)__popc(pm));
    base = __shfl_sync(am, base, leader);
    if (push) S.next_active[base + __popc(pm & ((1u << lane) - 1u))] = w;
}

__device__ __forceinline__ void flush_counts(const WalkOut &O, unsigned long long hops, unsigned long long bytes)
{
    hops = warp_sum(hops);
    bytes = warp_sum(bytes);
    if ((threadIdx.x & 31) == 0 && hops) {
        atomicAdd(&O.cnt->hops, hops);
        atomicAdd(&O.cnt->model_bytes, bytes);
    }
}

// solo tier: one thread per task (the task's walks, at most w_warp, in turn)
__global__ void __launch_bounds__(256) k_coop_solo(const WalkView V, const WalkOut O, const CoopState S,
                                                   const Task *tasks, unsigned n)
{
    unsigned long long hops = 0, bytes = 0;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const Task tk = tasks[i];
        int32_t g0, g1;
        node_groups(V, tk.node, g0, g1);
        for (int32_t k = 0; k < tk.count; k++) {
            const int32_t w = (int32_t)S.sorted_walks[tk.start + k];
            bool push;
            coop_hop(V, O, S, w, tk.node, g0, g1, nullptr, hops, bytes, push);
            if (push) {
                const unsigned slot = atomicAdd(S.n_next, 1u);
                S.next_active[slot] = w;
            }
        }
    }
    flush_counts(O, hops, bytes);
}

// warp tier: one warp per task; with SMEM the node's group timestamps go to
// the warp's slice of shared memory first
template <bool SMEM>
__global__ void __launch_bounds__(COOP_BLOCK) k_coop_warp(const WalkView V, const WalkOut O, const CoopState S,
                                                          const Task *tasks, unsigned n)
{
    __shared__ int64_t sts[SMEM ? BLOCK_G_CAP : 1];
    unsigned long long hops = 0, bytes = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned ti = blockIdx.x * COOP_WARPS + wid;
    if (ti < n) {
        const Task tk = tasks[ti];
        int32_t g0, g1;
        node_groups(V, tk.node, g0, g1);
        int64_t *mine = SMEM ? sts + wid * WARP_G_CAP : nullptr;
        if (SMEM) {
            for (int32_t g = lane; g < g1 - g0; g += 32) mine[g] = __ldg(V.ngts + g0 + g);
            __syncwarp();
        }
        const int32_t rounds = (tk.count + 31) / 32;
        for (int32_t rr = 0; rr < rounds; rr++) {
            const int32_t k = rr * 32 + lane;
            bool push = false;
            int32_t w = -1;
            if (k < tk.count) {
                w = (int32_t)S.sorted_walks[tk.start + k];
                coop_hop(V, O, S, w, tk.node, g0, g1, mine, hops, bytes, push);
            }
            push_active(S, push, w);
        }
    }
    flush_counts(O, hops, bytes);
}

// block tier: one block per (sub-)task
template <bool SMEM>
__global__ void __launch_bounds__(COOP_BLOCK) k_coop_block(const WalkView V, const WalkOut O, const CoopState S,
                                                           const Task *tasks, unsigned n)
{
    __shared__ int64_t sts[SMEM ? BLOCK_G_CAP : 1];
    unsigned long long hops = 0, bytes = 0;
    const Task tk = tasks[blockIdx.x];
    int32_t g0, g1;
        node_groups(V, tk.node, g0, g1);
    if (SMEM) {
        for (int32_t g = threadIdx.x; g < g1 - g0; g += blockDim.x) sts[g] = __ldg(V.ngts + g0 + g);
        __syncthreads();
    }
    const int32_t rounds = (tk.count + COOP_BLOCK - 1) / COOP_BLOCK;
    for (int32_t r = 0; r < rounds; r++) {
        const int32_t k = r * COOP_BLOCK + threadIdx.x;
        bool push = false;
        int32_t w = -1;
        if (k < tk.count) {
            w = (int32_t)S.sorted_walks[tk.start + k];
            coop_hop(V, O, S, w, tk.node, g0, g1, SMEM ? sts : nullptr, hops, bytes, push);
        }
        push_active(S, push, w);
    }
    flush_counts(O, hops, bytes);
}

// ---------------------------------------------------------------------------
// Hop-synchronous form for graph capture: one kernel per hop over the active
// list, whose length it reads from device memory, so the whole hop loop is a
// fixed sequence of launches with no host decision between them.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_graph_hop(const WalkView V, const WalkOut O, CoopState S,
                                                   const int32_t *__restrict__ active,
                                                   const unsigned int *__restrict__ n_active)
{
    unsigned long long hops = 0, bytes = 0;
    const int64_t n = *n_active;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t rounds = (n + stride - 1) / stride;
    for (int64_t r = 0; r < rounds; r++) {
        const int64_t i = r * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        bool push = false;
        int32_t w = -1;
        if (i < n) {
            w = active[i];
            const int32_t v = S.ws_node[w];
            int32_t g0, g1;
            node_groups(V, v, g0, g1);
            coop_hop(V, O, S, w, v, g0, g1, nullptr, hops, bytes, push);
        }
        push_active(S, push, w);
    }
    flush_counts(O, hops, bytes);
}

// Records the hop loop of one walk call on the stream (start kernel, then
// cap - 1 hop kernels alternating the two active lists, each preceded by a
// reset of the list it fills).  Used under stream capture.
static void record_graph_walk(tempest_t *h, const WalkView &V, const WalkOut &O, int64_t grid)
{
    cudaStream_t st = h->stream;
    unsigned int *ctr = h->co_ctr.as<unsigned int>();  // ctr[0], ctr[1]: active counts
    CoopState S;
    S.ws_node = h->co_node.as<int32_t>();
    S.ws_t = h->co_t.as<int64_t>();
    S.ws_len = h->co_len.as<int32_t>();
    S.ws_prev = h->co_prev.as<int32_t>();
    S.sorted_walks = nullptr;
    S.next_active = h->co_act[0].as<int32_t>();
    S.n_next = ctr;
    cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned int), st);
    k_coop_start<<<(unsigned)grid, 256, 0, st>>>(V, O, S);
    // cap - 1 hop kernels: a walk gains at most one node per kernel and a
    // PER_NODE walk starts with one (edge starts begin with two; their last
    // kernel then finds an empty list)
    for (int32_t step = 0; step + 1 < O.cap; step++) {
        const int src = step & 1, dst = src ^ 1;
        S.next_active = h->co_act[dst].as<int32_t>();
        S.n_next = ctr + dst;
        cudaMemsetAsync(ctr + dst, 0, sizeof(unsigned int), st);
        k_graph_hop<<<(unsigned)grid, 256, 0, st>>>(V, O, S, h->co_act[src].as<int32_t>(), ctr + src);
    }
}

int graph_run(tempest_t *h, const WalkView &V, const WalkOut &O, int64_t &launches)
{
    const int64_t n = O.n_walks;
    if (n >= (int64_t)INT32_MAX) return fail(h, TEMPEST_EINVAL, "graph walks: n_walks must be < 2^31");
    int rc;
    const size_t nz = (size_t)(n > 0 ? n : 1);
    if ((rc = ensure(h, h->co_node, sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_t, sizeof(int64_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_len, sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_prev, sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_act[0], sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_act[1], sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_ctr, 64 * sizeof(unsigned int)))) return rc;
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_graph_hop, 256, 0);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    int64_t grid = (int64_t)h->num_sms * blocks_per_sm;
    if (grid > (n + 255) / 256) grid = (n + 255) / 256;
    if (grid < 1) grid = 1;

    // capture the hop loop; update the cached executable graph when only the
    // kernel arguments changed, otherwise instantiate a new one
    cudaStream_t cap_stream = h->stream;
    bool own_stream = false;
    if (cap_stream == nullptr || cap_stream == cudaStreamLegacy) {
        // the legacy stream cannot be captured: record on a private stream
        if ((rc = cuda_check(h, cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking), "graph stream")))
            return rc;
        own_stream = true;
    }
    cudaStream_t saved = h->stream;
    h->stream = cap_stream;
    cudaGraph_t graph = nullptr;
    rc = cuda_check(h, cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (!rc) {
        record_graph_walk(h, V, O, grid);
        rc = cuda_check(h, cudaStreamEndCapture(cap_stream, &graph), "end capture");
    }
    h->stream = saved;
    if (!rc) {
        bool updated = false;
        if (h->graph_exec && h->graph_cap == O.cap) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(h->graph_exec, graph, &info) == cudaSuccess) updated = true;
            else cudaGetLastError();
        }
        if (!updated) {
            if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
            rc = cuda_check(h, cudaGraphInstantiate(&h->graph_exec, graph, 0), "graph instantiate");
            h->graph_cap = O.cap;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (!rc) {
        if (own_stream) {
            // keep stream order with the caller's (legacy) stream
            rc = cuda_check(h, cudaGraphLaunch(h->graph_exec, saved), "graph launch");
        } else {
            rc = cuda_check(h, cudaGraphLaunch(h->graph_exec, cap_stream), "graph launch");
        }
    }
    if (own_stream) cudaStreamDestroy(cap_stream);
    launches += 1 + (O.cap > 1 ? O.cap - 1 : 0);
    h->graph_launches++;
    return rc;
}

static int bits_for_n(int64_t N)
{
    int b = 0;
    while (b < 62 && ((N > 0 ? N - 1 : 0) >> b) != 0) b++;
    return b < 1 ? 1 : b;
}

int coop_run(tempest_t *h, const WalkView &V, const WalkOut &O, int64_t &launches)
{
    cudaStream_t st = h->stream;
    const int64_t n = O.n_walks;
    if (n >= (int64_t)INT32_MAX) return fail(h, TEMPEST_EINVAL, "cooperative walks: n_walks must be < 2^31");
    int rc;
    const size_t nz = (size_t)(n > 0 ? n : 1);
    if ((rc = ensure(h, h->co_node, sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_t, sizeof(int64_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_len, sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_prev, sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_act[0], sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_act[1], sizeof(int32_t) * nz, true))) return rc;
    if ((rc = ensure(h, h->co_runs, sizeof(int32_t) * 2 * nz, true))) return rc;
    const int64_t tier_stride = n + n / 8 + 64;
    if ((rc = ensure(h, h->co_tasks, sizeof(Task) * (size_t)(T_COUNT * tier_stride), true))) return rc;
    if ((rc = ensure(h, h->co_ctr, 64 * sizeof(unsigned int)))) return rc;
    for (int b = 0; b < 2; b++) {
        if ((rc = ensure(h, h->sk32[b], sizeof(uint32_t) * nz, true))) return rc;
        if ((rc = ensure(h, h->sv[b], sizeof(uint32_t) * nz, true))) return rc;
    }
    if ((rc = ensure(h, h->partials, sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 2)))) return rc;
    if ((rc = ensure(h, h->hist, sizeof(uint32_t) * (size_t)SORT_HIST_WORDS))) return rc;

    unsigned int *ctr = h->co_ctr.as<unsigned int>();  // [0..4] tier counts, [8] next active count
    unsigned int *hc = static_cast<unsigned int *>(h->hstat);
    CoopState S;
    S.ws_node = h->co_node.as<int32_t>();
    S.ws_t = h->co_t.as<int64_t>();
    S.ws_len = h->co_len.as<int32_t>();
    S.ws_prev = h->co_prev.as<int32_t>();
    int cur = 0;
    S.next_active = h->co_act[cur].as<int32_t>();
    S.n_next = ctr + 8;
    S.sorted_walks = nullptr;

    // step 0: start edges
    cudaMemsetAsync(ctr, 0, 64 * sizeof(unsigned int), st);
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)h->num_sms * 16) g = (int64_t)h->num_sms * 16;
    k_coop_start<<<(unsigned)(g > 0 ? g : 1), 256, 0, st>>>(V, O, S);
    launches++;
    cudaMemcpyAsync(hc, ctr + 8, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "coop start"))) return rc;
    int64_t n_active = hc[0];
    const int bits = bits_for_n(h->N);
    const int32_t w_warp = h->coop_w_warp, mega = h->coop_mega;

    while (n_active > 0) {
        const int32_t *active = h->co_act[cur].as<int32_t>();
        // 1. regroup: sort active walks by current node
        ActiveKeyLoader ld{active, S.ws_node};
        uint32_t *kb[2] = {h->sk32[0].as<uint32_t>(), h->sk32[1].as<uint32_t>()};
        uint32_t *vb[2] = {h->sv[0].as<uint32_t>(), h->sv[1].as<uint32_t>()};
        int sl = 0;
        const int r = radix_sort_launch<uint32_t>(ld, n_active, bits, kb, vb, h->hist.as<uint32_t>(), st, &sl);
        launches += sl;
        // 2. runs of equal nodes
        int32_t *run_pos = h->co_runs.as<int32_t>();
        int32_t *run_node = run_pos + n_active;
        RunOp op{kb[r], run_pos, run_node};
        const int nb = scan_launch(op, n_active, h->partials.as<uint64_t>(), st);
        launches += 3;
        // 3. classify into tiers
        cudaMemsetAsync(ctr, 0, 64 * sizeof(unsigned int), st);
        int64_t cg = (n_active + 255) / 256;
        if (cg > (int64_t)h->num_sms * 16) cg = (int64_t)h->num_sms * 16;
        k_coop_classify<<<(unsigned)cg, 256, 0, st>>>(run_pos, run_node, h->partials.as<uint64_t>() + nb, n_active,
                                                     V.ngr, w_warp, mega, h->co_tasks.as<Task>(), tier_stride,
                                                     ctr);
        launches++;
        cudaMemcpyAsync(hc, ctr, 8 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
        if ((rc = cuda_check(h, cudaStreamSynchronize(st), "coop classify"))) return rc;  // host sync 1
        unsigned cnt[T_COUNT];
        for (int t = 0; t < T_COUNT; t++) cnt[t] = hc[t];
        // 4. terminal kernels
        const int nxt = cur ^ 1;
        S.sorted_walks = vb[r];
        S.next_active = h->co_act[nxt].as<int32_t>();
        const Task *tk = h->co_tasks.as<Task>();
        if (cnt[T_SOLO])
            k_coop_solo<<<(cnt[T_SOLO] + 255) / 256, 256, 0, st>>>(V, O, S, tk + T_SOLO * tier_stride, cnt[T_SOLO]);
        if (cnt[T_WARP_SMEM])
            k_coop_warp<true><<<(cnt[T_WARP_SMEM] + COOP_WARPS - 1) / COOP_WARPS, COOP_BLOCK, 0, st>>>(
                V, O, S, tk + T_WARP_SMEM * tier_stride, cnt[T_WARP_SMEM]);
        if (cnt[T_WARP_GLOBAL])
            k_coop_warp<false><<<(cnt[T_WARP_GLOBAL] + COOP_WARPS - 1) / COOP_WARPS, COOP_BLOCK, 0, st>>>(
                V, O, S, tk + T_WARP_GLOBAL * tier_stride, cnt[T_WARP_GLOBAL]);
        if (cnt[T_BLOCK_SMEM])
            k_coop_block<true><<<cnt[T_BLOCK_SMEM], COOP_BLOCK, 0, st>>>(V, O, S, tk + T_BLOCK_SMEM * tier_stride,
                                                                        cnt[T_BLOCK_SMEM]);
        if (cnt[T_BLOCK_GLOBAL])
            k_coop_block<false><<<cnt[T_BLOCK_GLOBAL], COOP_BLOCK, 0, st>>>(
                V, O, S, tk + T_BLOCK_GLOBAL * tier_stride, cnt[T_BLOCK_GLOBAL]);
        for (int t = 0; t < T_COUNT; t++) launches += cnt[t] ? 1 : 0;
        for (int t = 0; t < T_COUNT; t++) h->coop_tier_launches[t] += cnt[t] ? 1 : 0;
        cudaMemcpyAsync(hc, ctr + 8, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
        if ((rc = cuda_check(h, cudaStreamSynchronize(st), "coop step"))) return rc;  // host sync 2
        n_active = hc[0];
        cur = nxt;
    }
    return TEMPEST_OK;
}

}  // namespace tw
