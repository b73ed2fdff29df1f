/*
 * tempest.h -- C ABI of the GB300 streaming temporal random-walk engine.
 *
 * The engine keeps a sliding window over a temporal edge stream in GPU
 * memory, indexes it two ways over one edge store, and draws causality-
 * preserving random walks from it (Tempest, Sec. 2).  Every call is a plain C
 * function taking plain pointers and sizes; no C++ or framework types cross
 * this boundary.
 *
 * Conventions
 *  - Every call returns a status: TEMPEST_OK (0) or a negative TEMPEST_E*
 *    code.  tempest_last_error() gives a human-readable reason.  No call
 *    aborts the process or leaves the handle half-updated on EINVAL.
 *  - Pointers to caller data may be host or device pointers; the library
 *    detects which (cudaPointerGetAttributes).  The caller keeps ownership.
 *    Host inputs are copied before the call returns.  Host outputs are
 *    complete when the call returns.  Device outputs are complete when work
 *    queued on the handle's stream before the next call has finished
 *    (stream order); tempest_sync() waits for it.
 *  - All device work runs on the stream given by tempest_set_stream (the
 *    legacy default stream when none is set).
 *  - Node ids are int32 >= 0; timestamps are int64.  The node arrays span
 *    [0, 1 + largest id ever ingested].  Live index entries (one per edge for
 *    directed graphs, two for undirected) must stay below 2^31 - 1.
 *  - The handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef TEMPEST_H
#define TEMPEST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tempest tempest_t;

enum {
    TEMPEST_OK = 0,
    TEMPEST_EINVAL = -1,    /* bad argument; no state changed */
    TEMPEST_ENOMEM = -2,    /* allocation failed or HBM budget exceeded */
    TEMPEST_ECUDA = -3,     /* a CUDA runtime call failed */
    TEMPEST_ETIMEDOUT = -4, /* reserved for a bounded device wait that gives up:
                             * no kernel of this library waits on a flag or a
                             * peer, so no call returns it */
    TEMPEST_EBUSY = -5      /* the serving queue is full */
};

/* Temporal bias of a hop (Sec. 2.5).  UNIFORM: every edge of Gamma_t(v)
 * equally likely (Eq. 1).  LINEAR: timestamp group i of Gamma_t(v), in
 * ascending time order, has weight i+1 (Eq. 2).  EXP: group i has weight
 * exp(lambda*i), drawn with the exact inverse CDF
 * x = n + log(u + (1-u) exp(-lambda n)) / lambda (Eq. 3 corrected: the printed
 * approximation cannot return the newest group).  For LINEAR and EXP an edge
 * is then drawn uniformly inside the chosen group (ties broken uniformly,
 * Sec. 2.1). */
enum { TEMPEST_BIAS_UNIFORM = 0, TEMPEST_BIAS_LINEAR = 1, TEMPEST_BIAS_EXP = 2,
       /* weight-based exponential (Sec. 2.5, the paper's default sampler):
        * every edge of Gamma_t(v) weighs exp(lambda_w (t_e - t_min)); an
        * inverse-CDF draw on the running weight (u1) picks the timestamp
        * group, an edge of it is uniform (u2).  A BIASED_TS start draws as
        * TEMPEST_BIAS_EXP does.  See tempest_set_weight_rate. */
       TEMPEST_BIAS_EXP_WEIGHT = 3,
       /* Temporal Node2Vec (Sec. 2.5): a hop from v, reached from u, draws
        * proposals from the TEMPEST_BIAS_EXP sampler over Gamma_t(v) and
        * accepts one with probability beta(u, w) / beta_max: beta = 1/p when
        * w is u, 1 when a live edge u -> w exists (either orientation for
        * undirected graphs; w -> u for backward walks), 1/q otherwise;
        * beta_max = max(1/p, 1, 1/q).  Proposal k of a hop uses Philox
        * counter (hop, k, walk) (proposal 0 is the exponential draw), its
        * acceptance uniform u = (r0:r1 >> 11) 2^-53 of counter (hop, 2^31 +
        * k, walk), accepted when u * beta_max < beta (drawn only when beta <
        * beta_max).  After TEMPEST_N2V_MAX_TRIALS rejections the walk ends.
        * The first hop of a PER_NODE walk has no u and takes proposal 0.
        * Starts draw as TEMPEST_BIAS_EXP.  See tempest_set_node2vec. */
       TEMPEST_BIAS_NODE2VEC = 4 };
#define TEMPEST_N2V_MAX_TRIALS 4096

/* Start selection (Sec. 2.3, timestamp-grouped view; Sec. 3 workloads).
 * UNIFORM_EDGE: a live edge uniformly.  BIASED_TS: a timestamp group of the
 * whole window under the walk's own bias (EXP uses the start rate), then an
 * edge uniformly inside the group.  PER_NODE: K walks from every active node
 * (a node with at least one live entry in the node view), in increasing id
 * order: walk w starts at active node w / K, K = n_walks / (active nodes),
 * which must divide; its first hop may take any of the node's live edges
 * (as from a time before every live edge) and uses Philox counter 0. */
enum { TEMPEST_START_UNIFORM_EDGE = 0, TEMPEST_START_BIASED_TS = 1, TEMPEST_START_PER_NODE = 2 };

/* Walk execution form (Sec. 2.4).  The result is the same for every form:
 * each walk draws from its own counter-based random stream. */
enum {
    TEMPEST_SCHED_FULL_WALK = 0, /* one thread carries one walk (Sec. 2.4.1) */
    TEMPEST_SCHED_COOP = 1,      /* per-hop regrouping by node, thread / warp /
                                    block tiers (Sec. 2.4.3-2.4.5, Alg. 1) */
    TEMPEST_SCHED_STREAM = 2     /* persistent lanes that refill from a
                                    work counter as walks end, one memory round
                                    trip per loop iteration, interpolation
                                    search of Gamma_t(v) (no counterpart in the
                                    paper: a GB300 form of Sec. 2.4.1) */,
    TEMPEST_SCHED_GRAPH = 3,     /* hop-synchronous: one kernel per hop over the
                                    active walks, the whole hop loop captured
                                    once as a CUDA graph and replayed */
    TEMPEST_SCHED_LANE = 4       /* default: persistent lanes that refill as
                                    walks end, each advancing one whole hop
                                    per loop iteration in lockstep with its
                                    warp */
};

/* Per-batch ingest report. */
typedef struct {
    int64_t n_in;          /* edges passed in */
    int64_t n_dropped_late;/* of those, older than the cut-off in force */
    int64_t n_evicted;     /* live edges removed by this batch's cut-off */
    int64_t n_live;        /* live edges after the batch */
    int64_t n_ts_groups;   /* distinct timestamps among live edges */
    int64_t n_node_groups; /* (node, timestamp) groups of the node view */
    int64_t n_nodes;       /* 1 + largest id seen */
    int64_t cutoff;        /* window cut-off (valid when has_cutoff) */
    int32_t has_cutoff;
    int32_t sorted_input;  /* the batch arrived in timestamp order */
    int64_t launches;      /* kernels this library launched for the batch */
    double evict_ms;       /* device time of the node view's eviction (the
                              per-node counts of the evicted edges and the
                              advance of each touched node's head), from CUDA
                              events on the handle's stream; the store and the
                              timestamp view evict by moving a head, O(1).  0
                              when nothing was evicted or the batch rebuilt
                              the node view (eviction is then part of it) */
    int64_t model_bytes;   /* algorithmic bytes of this batch in this library's
                              design: each array the batch touches (the batch,
                              the store append, the timestamp view's new
                              group starts, the evicted edges' ids and their
                              nodes' records, the node view's batch sort
                              passes, runs, region moves and scatter) read or
                              written once for its role; a full rebuild of
                              the node view counts its whole sort and
                              scatter over the live entries */
    int32_t view_rebuilt;  /* 1 when the batch rebuilt the node view whole */
    int32_t copied_ahead;  /* nodes that moved onto a copy of their live range
                            * made in the batches before (no whole slide) */
} tempest_ingest_stats;

/* Per-call walk report (valid once the call's work has finished). */
typedef struct {
    int64_t n_walks;
    int64_t hops;          /* edges traversed, start edge included */
    int64_t model_bytes;   /* sum of the per-hop sector model over the hops */
    int64_t launches;      /* kernels this library launched for the call */
    int64_t tier_launches[5]; /* TEMPEST_SCHED_COOP: terminal-kernel launches
                                 per tier (solo, warp-smem, warp-global,
                                 block-smem, block-global) */
    double kernel_ms;      /* device time of the walk kernels proper (start
                              draw and hops, without the row padding and
                              without the index preparation), from CUDA
                              events on the handle's stream; 0 if none ran */
    int64_t d2h_bytes;     /* bytes copied device to host for host outputs.
                              When node and ts are both host buffers, a
                              share of the rows (TEMPEST_TUNE_HOST_LINK_PCT)
                              is padded on the device and copied whole; the
                              others travel as their walks' cells, lengths
                              and offsets and host threads write their rows
                              and padding, overlapped with the first copy
                              when the caller's buffers are pinned (rows of
                              the band between them count where they went) */
    double host_ms[3];     /* that split's wall-clock phases (0 for other
                              outputs): [0] from the call's start until the
                              host part's cells, lengths and offsets are on
                              the host (walk kernels, padding, compaction and
                              their copies), [1] the host threads writing
                              their rows and padding, [2] the wait after
                              that for the copy of the rows padded on the
                              device */
} tempest_walk_stats;

/* Create an engine.  window > 0: duration Delta in timestamp units, the
 * active set is {e : t - Delta <= t_e <= t} with t the largest timestamp
 * ingested (Sec. 2.6).  window < 0: keep the -window newest edges, cutting at
 * the timestamp of the (-window)-th newest and keeping that whole timestamp
 * group.  window == 0: keep everything.  directed == 0 indexes every edge
 * under both endpoints.  *out receives the handle.  EINVAL on out == NULL. */
int tempest_create(int64_t window, int directed, tempest_t **out);

/* Free the handle and all device memory it owns.  NULL is accepted. */
int tempest_destroy(tempest_t *h);

/* Rate lambda_w > 0 (per timestamp unit) of the weight-based sampler
 * (TEMPEST_BIAS_EXP_WEIGHT; default 1e-9, i.e. per second for nanosecond
 * timestamps).  Group weights are kept in the index from the first call of
 * this function or the first weight-based walk on, at a cost per ingested
 * group; the first walk call after a change recomputes all of them.  EINVAL
 * on lambda_w <= 0 or not finite. */
int tempest_set_weight_rate(tempest_t *h, double lambda_w);

/* Return parameter p and in-out parameter q of Temporal Node2Vec walks
 * (TEMPEST_BIAS_NODE2VEC; default 1, 1).  With q != 1 the neighbour test
 * matters: the handle builds a table of the live (from, to) pairs now (about
 * 64 bytes per live edge) and every ingest keeps it current.  EINVAL unless
 * 1e-3 <= p, q <= 1e3; ENOMEM when the table does not fit. */
int tempest_set_node2vec(tempest_t *h, double p, double q);

/* Queue all further device work of the handle on stream (a cudaStream_t). */
int tempest_set_stream(tempest_t *h, void *stream);

/* Route device allocations through alloc(bytes, ctx) / release(ptr, ctx)
 * (e.g. a framework's caching allocator) and cap the handle's device memory
 * at hbm_budget bytes (0 = no cap).  Either callback may be NULL to restore
 * cudaMalloc / cudaFree.  alloc must return device memory aligned to 256
 * bytes, as cudaMalloc does (a call that gets another pointer releases it
 * and fails with EINVAL, the handle unchanged).  Call before the first
 * ingest. */
int tempest_set_allocator(tempest_t *h, void *(*alloc)(size_t bytes, void *ctx),
                          void (*release)(void *ptr, void *ctx), void *ctx, size_t hbm_budget);

/* Exponential rates: lambda_hop > 0 per timestamp group for hops (1 is the
 * paper's form); lambda_start > 0 for BIASED_TS start selection, or 0 for
 * 1 / (number of timestamp groups in the window), i.e. one e-fold across the
 * window.  EINVAL otherwise. */
int tempest_set_bias_params(tempest_t *h, double lambda_hop, double lambda_start);

/* Ingest one batch of n edges (Sec. 2.6): every edge gets the next arrival
 * index; edges older than the cut-off in force are dropped and counted; the
 * rest are sorted by timestamp (arrival order among ties) and merged into
 * the edge store; the cut-off advances and the edges before it are evicted;
 * both views are rebuilt (Sec. 2.3).  src, dst: int32[n] node ids >= 0;
 * ts: int64[n], each strictly between INT64_MIN (the time before every
 * edge, which walk outputs give their first node) and INT64_MAX (the time
 * after every edge, where PER_NODE backward walks start).  stats may be
 * NULL.  EINVAL (state unchanged) on n < 0, NULL arrays with n > 0, a
 * negative id or an INT64_MIN or INT64_MAX timestamp.  ENOMEM (a failed
 * allocation or the HBM budget) and ECUDA (a failed consistency check) also
 * leave the state as it was: the batch is not ingested (nor into the in-edge
 * index of backward walks), the edge store's counters are restored (its
 * previous live edges are still in place) and the derived views are rebuilt
 * from it, at once or, when that needs memory that is not there, before the
 * next call that reads them (which then returns ENOMEM itself while the
 * memory stays short).  Synchronises the stream. */
int tempest_ingest(tempest_t *h, const int32_t *src, const int32_t *dst, const int64_t *ts,
                   int64_t n, tempest_ingest_stats *stats);

/* Draw n_walks walks (Sec. 2.1, 2.4, 2.5).  Walk w uses Philox4x32-10
 * (Salmon et al., SC'11) with key = seed and counter (hop, 0, w_lo, w_hi);
 * the draw that appends the node at row position p uses hop = p - 1 (hop 0
 * selects the start edge, which gives positions 0 and 1; under PER_NODE it
 * is the first hop from the start node).  From each
 * block, u1 = (r0:r1 >> 11) * 2^-53 picks the edge or group and
 * u2 = (r2:r3 >> 11) * 2^-53 the edge inside a group; bit 0 of r3 orients an
 * undirected start edge.  At node v and time t the next edge comes from
 * Gamma_t(v) = {(v, w, t') : t' > t}; the walk stops when Gamma_t(v) is
 * empty or max_len nodes are reached.
 * Outputs, row-major with row stride max_len: node int32[n_walks*max_len],
 * ts int64[n_walks*max_len] (ts of node 0 is INT64_MIN; padding is node -1,
 * ts INT64_MIN), len int32[n_walks] (nodes written; 0 on an empty window).
 * The outputs may be device or host memory (each pointer is classified);
 * device outputs are written by the kernels in stream order, host outputs
 * are complete when the call returns (see tempest_walk_stats.d2h_bytes for
 * how they travel; pinned host buffers let the copy overlap the host-side
 * row writes).  EINVAL on n_walks < 0, max_len < 2, bad bias / start policy
 * or NULL outputs. */
int tempest_walks(tempest_t *h, int64_t n_walks, int32_t max_len, int bias, int start_policy,
                  uint64_t seed, int32_t *node, int64_t *ts, int32_t *len);

/* Backward walks (the walk form of tempest_enable_backward): arguments,
 * outputs and draw counters as in tempest_walks; node 0 -> node 1 is a start
 * edge walked from its destination to its source, and each later position
 * is an in-edge of the current node earlier than the current time.  Biases
 * 0-2.  EINVAL as tempest_walks, on bias 3, or on a directed graph without
 * tempest_enable_backward. */
int tempest_walks_backward(tempest_t *h, int64_t n_walks, int32_t max_len, int bias, int start_policy,
                           uint64_t seed, int32_t *node, int64_t *ts, int32_t *len);

/* Like tempest_walks with a per-walk length cap and bias, all in one launch:
 * max_len_arr int32[n_walks] (each in [2, max_len_cap]), bias_arr
 * uint8[n_walks] (each a TEMPEST_BIAS_*).  Rows have stride max_len_cap. */
int tempest_walks_mixed(tempest_t *h, int64_t n_walks, const int32_t *max_len_arr,
                        int32_t max_len_cap, const uint8_t *bias_arr, int start_policy,
                        uint64_t seed, int32_t *node, int64_t *ts, int32_t *len);

/* The closed-form samplers on their own (Sec. 2.5, Eq. 1-3): out[i] is the
 * index in [0, n[i]) that `bias` selects for the uniform u = u_bits[i] * 2^-53,
 * computed exactly as walk hops compute it.  u_bits: uint64[count], each
 * < 2^53; n: int64[count], each in [1, 2^31); out: int64[count]; all device
 * memory.  lambda > 0 is the exponential rate.  Queued on the handle's
 * stream.  EINVAL on a bad bias, lambda, count < 0 or non-device arrays. */
int tempest_sample_index(tempest_t *h, const uint64_t *u_bits, const int64_t *n, int64_t count, int bias,
                         double lambda, int64_t *out);

/* One walk request of a batched launch.  All pointers are device memory.
 * Rows have stride max_len; max_len_arr / bias_arr (nullable) give per-walk
 * caps (each in [2, max_len]) and biases.  Walk w of the request draws from
 * Philox(seed, w, hop) exactly as tempest_walks(n_walks, ..., seed) would, so
 * its result does not depend on the other requests of the launch. */
typedef struct {
    int64_t n_walks;
    int32_t max_len;
    int32_t bias;
    const int32_t *max_len_arr;
    const uint8_t *bias_arr;
    int32_t start_policy;
    int32_t direction;  /* 0: forward; 1: backward (see tempest_enable_backward) */
    uint64_t seed;
    int32_t *node;
    int64_t *ts;
    int32_t *len;
} tempest_walk_request;

/* Backward walks (Sec. 2.1, "the backward case defined analogously"): a
 * request with direction 1 walks the time-reversed graph, in which every
 * live edge (u, v, t) reads as (v, u, -t) in mirrored arrival order.  From
 * node v at time t it draws from the in-edges of v earlier than t,
 * {(u, v, t') : t' < t}, taken latest first (the samplers' index 0 is the
 * latest edge or group; the bias favours older ones as the forward bias
 * favours newer ones); a start edge (u, v, t) is walked from v to u, and a
 * PER_NODE start begins after every live edge.  Biases 0-2 only.  Directed
 * graphs need this call first: from it on every ingest also keeps an index
 * of the in-edges (a second store and view, built now from the live edges).
 * Undirected graphs walk backward on their one view.  ENOMEM when the
 * second index does not fit. */
int tempest_enable_backward(tempest_t *h);

/* Serve n_req walk requests in one persistent launch (continuous batching
 * of requests; Sec. 2.4 walks, Sec. 2.5 samplers).  The requests' outputs
 * are complete when the handle's stream reaches this point.  EINVAL on a
 * bad request (same rules as tempest_walks_mixed) or non-device pointers. */
int tempest_walks_batch(tempest_t *h, const tempest_walk_request *reqs, int n_req);

/* ---- serving loop (continuous batching over the device-resident index) ----
 * The paper runs one walk call per batch (Sec. 3.3); these calls serve a
 * stream of requests instead.  A server keeps a FIFO of ingest and walk
 * requests.  Walk requests are admitted in arrival order into a wave (one
 * tempest_walks_batch launch) while the wave has launch slots
 * (max_wave_walks) and their outputs fit in an output arena of arena_bytes
 * (the HBM budget for results; requests passing NULL outputs get arena
 * memory, which returns on tempest_server_release).  Up to max_inflight
 * (1 or 2) waves run at once on the server's own streams, so requests that
 * arrive while a wave runs start in the next wave and overlap it.  An ingest
 * waits until no wave is in flight, so every walk request sees the index as
 * of its arrival.  A wave is ordered after all work queued on the handle's
 * stream when it launches; caller-provided arrays must be ready by then.  Ingest arrays (device memory) must stay valid until the
 * request completes.  No call blocks except tempest_server_drain and the
 * ingest that tempest_server_progress runs.  State: 0 queued, 1 running,
 * 2 done, negative = failed with that TEMPEST_E* code (ENOMEM: the request's
 * outputs can never fit the arena). */
typedef struct tempest_server tempest_server_t;
int tempest_server_create(tempest_t *h, size_t arena_bytes, int64_t max_wave_walks, int max_inflight,
                          tempest_server_t **out);
int tempest_server_destroy(tempest_server_t *s);
int tempest_server_submit_walks(tempest_server_t *s, const tempest_walk_request *req, uint64_t *ticket);
int tempest_server_submit_ingest(tempest_server_t *s, const int32_t *src, const int32_t *dst, const int64_t *ts,
                                 int64_t n, uint64_t *ticket);
/* Retire finished waves, run a ready ingest, launch new waves; *n_completed
 * receives the number of requests that finished during the call. */
int tempest_server_progress(tempest_server_t *s, int *n_completed);
/* State, output pointers (device) and submit-to-completion latency in
 * seconds (-1 while unfinished) of a request. */
int tempest_server_status(tempest_server_t *s, uint64_t ticket, int *state, int32_t **node, int64_t **ts,
                          int32_t **len, double *latency_s);
/* Forget a finished request and return its arena memory. */
int tempest_server_release(tempest_server_t *s, uint64_t ticket);
/* Progress until the queue is empty and no wave runs. */
int tempest_server_drain(tempest_server_t *s);
/* out[0] waves launched, out[1] walk requests served in waves, out[2]
 * ingests run, out[3] requests queued. */
int tempest_server_stats(tempest_server_t *s, int64_t out[4]);

/* Select the walk execution form (TEMPEST_SCHED_*) for later walk calls. */
int tempest_set_scheduler(tempest_t *h, int mode);

/* Tuning knobs.  None of them changes a walk, only how fast it is drawn:
 * every setting gives bit-identical outputs.  Change them between walk calls
 * (not while a server wave is in flight). */
enum {
    /* log2 of the mean number of timestamp groups per time bucket of a node
     * with >= 32 groups (the hop search index, Sec. 2.3), 0..5; default 2 */
    TEMPEST_TUNE_BKT_LOG = 0,
    /* TEMPEST_SCHED_COOP: largest run of walks at one node served one thread
     * per walk (W_warp of Sec. 2.4.3), 1..256; default 4 */
    TEMPEST_TUNE_COOP_W_WARP = 1,
    /* TEMPEST_SCHED_COOP: walks per block sub-task of a mega-hub run
     * (Sec. 2.4.4), 256..2^30; default 8192 */
    TEMPEST_TUNE_COOP_MEGA = 2,
    /* TEMPEST_SCHED_STREAM: resident 256-thread CTAs per SM of the persistent
     * walker, 0 = as many as fit; values above 4 select a build with a
     * smaller register budget (more warps in flight, a few spills); 0..16;
     * default 0 */
    TEMPEST_TUNE_STREAM_CTAS = 3,
    /* TEMPEST_SCHED_LANE: 0 (default) the walker writes each row's padding
     * as its walk ends; 1 one streaming pass pads all rows after the walks */
    TEMPEST_TUNE_PAD_PASS = 4,
    /* walks into host buffers: percent of the rows padded on the device
     * (0-100, default 62); the others travel as their walks' cells only and
     * host threads write their rows and padding meanwhile.  Between 1 and 99
     * the padded rows are a band that the copy takes a chunk at a time from
     * below while the host threads, once their own rows are written, take it
     * from above (its cells travel too); 100 copies every row whole, 0 sends
     * every row as cells */
    TEMPEST_TUNE_HOST_LINK_PCT = 5,
    /* walks into host buffers: host threads that write the rows sent as
     * cells (0-256; 0, the default: the CPUs this process may run on, from
     * its affinity mask and cgroup CPU quota, at most 32) */
    TEMPEST_TUNE_HOST_THREADS = 6,
    /* ingest: how the node view finds what each node lost to eviction (Sec.
     * 2.6): 0 (default) chooses, 1 counts the evicted edges' endpoints, 2
     * has every active node search its own entries for the new store head
     * (chosen when the active nodes are fewer than an eighth of the evicted
     * entries) */
    TEMPEST_TUNE_EVICT = 7,
    /* ingest: live entries from which a node whose regions fill copies its
     * live range to their front a share per batch in the 16 batches before,
     * instead of in one batch, and live edges from which the store copies its
     * live range to its other buffer in the 6 batches before it fills (Sec.
     * 2.6 sliding window), 16..2^30; default 2^20 */
    TEMPEST_TUNE_MIRROR_MIN = 8
};
/* Set / read one knob.  EINVAL on an unknown knob or a value out of range. */
int tempest_set_tuning(tempest_t *h, int knob, int64_t value);
int tempest_get_tuning(tempest_t *h, int knob, int64_t *value);

#define TEMPEST_TUNE_MAX_TRIALS 48
typedef struct {
    int32_t sched, bkt_log, coop_w_warp, coop_mega, stream_ctas, pad_pass;
    double ms;             /* walk-call device time (start to padded rows) */
} tempest_tune_trial;
typedef struct {
    int32_t sched, bkt_log, coop_w_warp, coop_mega, stream_ctas, pad_pass; /* chosen */
    int32_t n_trials, reserved;
    double best_ms;        /* call time of the chosen configuration */
    double start_ms;       /* call time of the configuration it started from */
    tempest_tune_trial trials[TEMPEST_TUNE_MAX_TRIALS];
} tempest_tune_report;
#define TEMPEST_TUNE_FORMS 1       /* flags: also choose the walk form */
#define TEMPEST_TUNE_PER_INGEST 2  /* flags: every timed call also rebuilds the
                                      derived walk indexes (time buckets,
                                      active nodes, weight sums), as the first
                                      walk call after an ingest does */

/* Autotuner: times walk calls of n_walks walks (max_len, bias, start_policy,
 * seed as in tempest_walks) on the current index state for candidate
 * settings, by coordinate descent: the walk form (with TEMPEST_TUNE_FORMS),
 * then the bucket density, then the chosen form's own knobs (CTAs per SM for
 * the streaming form; W_warp then the mega-hub split for the cooperative
 * form).  Each candidate is timed with CUDA events on the handle's stream as
 * the minimum of 3 calls after one warm-up call; outputs go to scratch
 * memory the handle owns.  The best setting stays selected on the handle
 * and is described in *out (nullable).  Blocking; EINVAL on bad arguments. */
int tempest_autotune(tempest_t *h, int64_t n_walks, int32_t max_len, int bias, int start_policy, uint64_t seed,
                     int32_t flags, tempest_tune_report *out);

/* The same, timing tempest_walks_mixed calls on the caller's own per-walk
 * lengths and biases (device arrays of n_walks, as in tempest_walks_mixed),
 * so a mixed workload is tuned on its own mix. */
int tempest_autotune_mixed(tempest_t *h, int64_t n_walks, const int32_t *max_len_arr, int32_t max_len_cap,
                           const uint8_t *bias_arr, int start_policy, uint64_t seed, int32_t flags,
                           tempest_tune_report *out);

/* Number of active nodes (nodes with at least one live entry in the node
 * view) of the current state: the divisor of PER_NODE walk counts. */
int tempest_active_nodes(tempest_t *h, int64_t *n);

/* The same for backward walks: nodes with at least one live in-edge (any
 * live edge, for undirected graphs).  EINVAL on a directed graph without
 * tempest_enable_backward. */
int tempest_active_nodes_backward(tempest_t *h, int64_t *n);

/* Report of the most recent walk call; waits for its work to finish. */
int tempest_last_walk_stats(tempest_t *h, tempest_walk_stats *out);

/* Live counters: out[0..9] = live edges m, timestamp groups, n_nodes, node
 * view entries M, node groups, dropped-late total, evicted total, has_cutoff,
 * cutoff, next arrival index. */
int tempest_get_counts(tempest_t *h, int64_t out[10]);

/* Export one array of the index state into dst (host or device) for
 * checking: which = TEMPEST_STATE_*.  cap is dst's capacity in elements;
 * *n receives the element count (call with dst == NULL to query it).  The
 * arrays are the canonical forms of Sec. 2.3: the live store in (ts, arrival)
 * order, the start offset of every timestamp group plus m, per node the start
 * of its segment of the node view plus M, the node view as store slots
 * (position, or 2*position + side for undirected graphs), the start of every
 * (node, timestamp) group plus M, and per node its first group index. */
enum {
    TEMPEST_STATE_SRC = 0,            /* int32[m]   */
    TEMPEST_STATE_DST = 1,            /* int32[m]   */
    TEMPEST_STATE_TS = 2,             /* int64[m]   */
    TEMPEST_STATE_TS_GROUP_OFF = 3,   /* int32[G+1] */
    TEMPEST_STATE_NODE_OFF = 4,       /* int32[N+1] */
    TEMPEST_STATE_NODE_ORDER = 5,     /* int32[M]   */
    TEMPEST_STATE_NODE_GROUP_OFF = 6, /* int32[Gn+1] */
    TEMPEST_STATE_NODE_GIDX = 7       /* int32[N+1] */
};
int tempest_export_state(tempest_t *h, int which, void *dst, int64_t cap, int64_t *n);

/* Wait for all work queued on the handle's stream. */
int tempest_sync(tempest_t *h);

/* Reason for the last failing call on h (or of tempest_create when h is
 * NULL).  Valid until the next call on h. */
const char *tempest_last_error(tempest_t *h);

/* Library version string. */
const char *tempest_version(void);

/* Allocation-free batch sort.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory at run time -- code
 * under a fixed memory plan (a host framework that owns every device byte
 * through its own pool) or a latency-critical loop that cannot afford
 * cudaMalloc's implicit synchronisation.
 *
 * Sorts n edges by timestamp, keeping arrival order among equal timestamps
 * (the batch sort that begins every ingest), and writes the sorted batch to
 * out_src / out_dst / out_ts.  All six arrays must be device memory
 * (int32[n], int32[n], int64[n] each); the work is queued on `stream` (a
 * cudaStream_t, NULL for the legacy stream) and the call does not wait for it.
 * Scratch is a static device array of TEMPEST_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits; nothing is
 * allocated or freed.  The first call on a device looks up that array's
 * device address, so make it before any stream capture; the address is
 * looked up again when the device's context has changed since (after a
 * cudaDeviceReset), so call it again outside a capture then.  All calls share the
 * array: calls whose work overlaps on the GPU race.  Returns EINVAL (see
 * tempest_last_error(NULL)) for n < 0, n > TEMPEST_NOALLOC_MAX_EDGES or a
 * non-device array; n == 0 does nothing. */
#define TEMPEST_NOALLOC_MAX_EDGES 262144
#define TEMPEST_NOALLOC_SCRATCH_BYTES 6815744
int tempest_sort_batch_noalloc(const int32_t *src, const int32_t *dst, const int64_t *ts, int64_t n,
                               int32_t *out_src, int32_t *out_dst, int64_t *out_ts, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TEMPEST_H */
