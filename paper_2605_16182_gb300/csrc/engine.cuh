// engine.cuh -- the engine handle and the internal interfaces between the
// C ABI (capi.cu), ingest (ingest.cu) and walk generation (walks.cu).
#pragma once

#include <chrono>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tempest.h"

namespace tw {

// One entry of the node-and-timestamp-grouped view (Sec. 2.3).  The paper's
// view is offsets over the shared store; here each entry also carries the
// timestamp and the far endpoint of its edge, so a hop reads one 16-byte
// aligned record instead of chasing a store position into two more arrays.
struct __align__(16) Entry {
    int64_t ts;
    int32_t other;  // the endpoint a hop moves to
    int32_t slot;   // store position (directed) or 2*position + side
};

struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

// Small device-side record the ingest kernels fill and the host reads back.
struct IngestScratch {
    long long ts_min, ts_max;
    int max_id, neg_id;  // neg_id: bit 0 a negative id, bit 1 an INT64_MIN, bit 2 an INT64_MAX timestamp
    unsigned long long late, unsorted;
    long long cut;          // new cut-off
    int has_cut, pad0;
    long long i0, j0;       // first kept store / batch element
    long long kept_batch_min_ts;
    long long store_last_ts;
    long long tg_lo, tg_added;  // timestamp view: first live group, groups appended
    unsigned long long status;  // nonzero: an index check failed (bit per site)
};

// The per-node record a hop reads first: the node's live groups [g_lo,
// g_hi), its time-bucket table (nodes with enough groups; set when the
// tables are built: tb the table's first entry, bs the bucket width's log2
// in the low 6 bits and the build's generation above them), and the
// timestamps of its first and last live groups.  32 bytes, one sector: a
// hop gets everything it needs before the search in one round trip.
struct __align__(32) NodeRange {
    int32_t g_lo, g_hi;
    int32_t tb, bs;
    int64_t t_first, t_last;
};

// Device counters of the node-view update (one batch).
struct NvCounters {
    unsigned long long e_top, g_top;  // pool bump pointers
    long long gn_delta;               // groups added - groups removed
    unsigned long long n_ev_nodes;    // nodes that lost entries
    unsigned long long n_reloc;       // regions to move
    unsigned long long n_act;         // nodes owning regions
    unsigned long long overflow;      // a pool could not serve a region
    unsigned long long status;        // nonzero: a consistency check failed
    unsigned long long n_dense;       // batch-local node ids handed out
    unsigned long long w_rebase;      // a group weight's exponent grew too large
    unsigned long long moved_e;       // live entries of the regions that move (a batch's report)
    unsigned long long moved_g;       // live groups of the regions that move
    unsigned long long g_added;       // groups the batch adds
    unsigned long long ev_removed;    // entries the per-node eviction search removed
    unsigned long long mir_switched;  // nodes that moved onto their copy made ahead (group weights go stale)
};

// What the node view did for one batch: the counts its algorithmic-bytes
// model needs (see ingest_model_bytes).
struct NvBatchReport {
    int64_t ev_entries = 0, ev_nodes = 0;              // evicted entries and the nodes that lost them
    int64_t ev_scanned = 0;                             // active nodes searched instead of counting (0: counted)
    int64_t copied_ahead = 0;                           // nodes moved onto a copy made ahead
    int64_t entries = 0, ids = 0, passes = 0, runs = 0;  // appended entries, distinct nodes, sort passes, node runs
    int64_t moved_e = 0, moved_g = 0, g_added = 0;     // region moves; groups added
    bool rebuilt = false;                               // the whole view was rebuilt instead
    int64_t rb_entries = 0, rb_passes = 0, rb_nodes = 0, rb_groups = 0;
};

// A region move: live entries and groups of one node to fresh regions.
struct Reloc {
    int32_t old_e, n_e, new_e;
    int32_t old_g, n_g, new_g;
};

// A big node's copy of its live range to the front of its own regions, made
// a share per batch ahead of the batch that no longer fits: entries from
// x_m and groups from g_m, c_e / c_g of them copied so far (node -1: free).
struct NvMirror {
    int32_t node, x_m, g_m, c_e, c_g, pad0, pad1, pad2;
};

// Device-side walk counters.
struct WalkCounters {
    unsigned long long hops;
    unsigned long long model_bytes;
    unsigned long long status;  // nonzero: a kernel found corrupt state
    unsigned long long pad;
};

}  // namespace tw

struct tempest {
    // configuration
    int64_t window = 0;
    int directed = 1;
    double lam_hop = 1.0;
    double lam_start = 0.0;  // 0: 1 / G_tot
    double lam_w = 1e-9;     // weight-based sampler rate per timestamp unit
    int sched = TEMPEST_SCHED_LANE;
    int pad_pass = 0;  // lane walker: 1 pads rows in one pass after the walks
    cudaStream_t stream = nullptr;
    void *(*alloc_fn)(size_t, void *) = nullptr;
    void (*release_fn)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    size_t budget = 0;
    size_t in_use = 0;
    int device = 0;
    int num_sms = 1;

    // host mirror of the live state's sizes and counters
    int64_t m = 0;      // live edges
    int64_t G = 0;      // timestamp groups
    int64_t N = 0;      // node slots (1 + max id seen)
    int64_t M = 0;      // node view entries
    int64_t Gn = 0;     // node groups
    int64_t dropped = 0, evicted = 0, seq_next = 0;
    int has_cutoff = 0;
    int64_t cutoff = 0;

    // edge store: SoA buffers (two, for compaction and general merges).  The
    // live edges are buffer indices [s_lo, s_hi) of buffer cur, in (ts,
    // arrival) order; eviction advances s_lo, an append writes at s_hi.  The
    // absolute position of index i is s_base + i (node view slots hold it
    // modulo 2^32, so a compaction that moves the live range to index 0 only
    // changes s_base).
    tw::DBuf st_src[2], st_dst[2], st_ts[2];
    int cur = 0;
    int64_t s_lo = 0, s_hi = 0, s_cap = 0, s_base = 0;
    // store pre-copy: while on, the other buffer holds the absolute positions
    // [smir_a0, smir_done) at index position - smir_a0, so that the move to it
    // when the current buffer fills copies only what the last batches added
    bool smir_on = false;
    int64_t smir_a0 = 0, smir_done = 0;
    // timestamp-view pre-copy, the same for the group starts: while on, tg2
    // holds the positions [tmir_a0, tmir_done) of tg at index position -
    // tmir_a0; tg_lo_step: groups the last batch evicted from the view
    bool tmir_on = false;
    int64_t tmir_a0 = 0, tmir_done = 0, tg_lo_step = 0;
    // timestamp-grouped view: absolute store position (modulo 2^32) of the
    // start of every group, live groups [tg_lo, tg_hi) with tg[tg_hi] the
    // absolute end; the first live group may start before the head (its
    // evicted part is skipped on read)
    tw::DBuf tg, tg2;  // int32; tg2 receives tg when it moves to a larger buffer
    int64_t tg_lo = 0, tg_hi = 0;
    // node view in a slack layout: every node with entries owns a region of
    // the entry pool and one of the group pools, with room to grow; the
    // groups of node v are [ngr[v].x, ngr[v].y), group g's entries start at
    // ngo[g] and the slot after the node's last group holds its entry end
    tw::DBuf ent;   // Entry pool
    tw::DBuf ngo;   // int32 group start (entry pool index)
    tw::DBuf ngts;  // int64 group timestamp
    tw::DBuf ngr;   // NodeRange [N+1]
    tw::DBuf nrec;  // int4 [N+1]: entries [x, y), entry region end z, group region end w
    tw::DBuf nbeg;  // int2 [N+1]: entry region begin x, group region begin y
    tw::DBuf act;   // int32: nodes that own regions
    tw::DBuf nvc;   // device counters of the node view (NvCounters)
    int64_t n_act = 0;
    int64_t nrec_n = 0;     // node slots the per-node arrays cover
    int64_t e_cap = 0, g_cap = 0;
    int nv_shift = 0;       // region capacity = x + (x >> nv_shift) + 16
    bool nv_ready = false;
    tw::DBuf nv_tmp, run_node, run_pos, run_g, run_of, fx, run_de, run_dg, ev_nodes, reloc;
    tw::DBuf dense;    // int32 [N+1]: 1 + a batch-local id of each node the batch touches (0 between batches)
    // weight-based sampler: per-group weights (group size * exp(lam_w (t_g -
    // wref[v]))) kept by ingest once enabled, and per-node suffix sums of them
    // built for the walks of a state version
    tw::DBuf gw, gs;   // double, group pool indexing
    tw::DBuf wref;     // int64 [N+1] per-node reference time
    tw::DBuf w_cbase, w_ctot, w_coff;  // suffix-sum chunk lists
    bool w_on = false;     // weights are maintained
    bool w_valid = false;  // every live group's weight is current
    int64_t w_ver = -1;    // state version of the suffix sums
    tw::DBuf touched;  // int32: node of each batch-local id
    tw::DBuf ent_tmp;  // Entry: a batch's node view entries in (node, ts, arrival) order
    tw::DBuf nv_flags; // uint8 per batch entry: run start (bit 0), group start (bit 1)
    tw::DBuf nv_tex;   // uint64 per BSCAN_TILE batch entries: runs (high) and groups (low) before the tile
    tw::DBuf nv_mir;   // NvMirror[NV_MIRRORS]: big nodes copying their live range ahead of a slide
    int64_t S = 0;     // nodes that own regions (for the bucket index)
    int64_t state_ver = 0;  // bumped by every ingest
    // an ingest that failed after changing the store restored the store's
    // counters; the views (and the pair table) are rebuilt from the store
    // before their next use
    bool views_dirty = false;
    tw::NvBatchReport nv_rep;  // the node view's part of the last batch

    // time buckets of high-degree nodes (built lazily for the walks of a
    // state version): per node its table base, the tables, the big-segment
    // list and its chunk prefix
    tw::DBuf bkt;        // int32 tables (each big node's base is in its NodeRange)
    tw::DBuf big_node, big_t, big_c, big_own;
    tw::DBuf big_aux0, big_aux1, big_bf;  // per big node: build plan (int4, int4) and first bucket (int64)
    tw::DBuf bkt_prev;                    // the previous build's tables, the source of the next build's copies
    tw::DBuf nev;                         // int32 [N+1]: groups each node has lost to eviction (mod 2^32)
    int bkt_gen = 0;                      // build generation (the tables in bkt)
    bool bkt_prev_ok = false;             // bkt_prev holds generation bkt_gen - 1 of the current group numbering
    int64_t bkt_ver = -1;
    // active nodes in id order, for PER_NODE starts (built lazily per state)
    tw::DBuf pn_nodes;
    int64_t n_pn = 0;
    int64_t pn_ver = -1;
    int64_t n_big = 0;
    int bkt_log = 2;     // log2 of the mean groups per bucket

    // scratch
    tw::DBuf b_src, b_dst, b_ts;     // batch staged from host
    tw::DBuf b_gflag;                // uint8 per batch edge: its timestamp differs from the edge before it
    tw::DBuf sb_src, sb_dst, sb_ts;  // batch sorted by timestamp
    tw::DBuf sk64[2], sk32[2], sv[2];
    tw::DBuf hist, partials;
    tw::DBuf ev;                 // int32 [N+1] per-node evicted entries (zero between batches)
    // cooperative scheduler: walk state, active lists, runs, tier tasks, counters
    tw::DBuf co_node, co_t, co_len, co_prev, co_act[2], co_runs, co_tasks, co_ctr;
    int coop_w_warp = 4;         // solo / warp boundary W_warp (Sec. 3.5)
    int coop_mega = 8192;        // mega-hub split (Sec. 2.4.4)
    int stream_ctas = 0;         // persistent walker CTAs per SM (0: occupancy limit)
    tw::DBuf tune_out;           // autotuner walk outputs
    int64_t coop_tier_launches[5] = {0, 0, 0, 0, 0};
    cudaGraphExec_t graph_exec = nullptr;  // captured hop loop (TEMPEST_SCHED_GRAPH)
    int32_t graph_cap = 0;
    int64_t graph_launches = 0;
    tw::DBuf dstat;       // IngestScratch
    tw::DBuf wcnt;        // WalkCounters
    tw::DBuf out_stage;   // device staging of host walk outputs
    tw::DBuf in_stage;    // device staging of host walk inputs
    tw::DBuf exp_stage;   // export staging
    void *hstat = nullptr;     // pinned host mirror of IngestScratch / counters
    // walks into host buffers: rows are compacted on the device, copied, and
    // expanded on the host (pinned host staging, grown as needed)
    void *hpin = nullptr;
    size_t hpin_bytes = 0;
    tw::DBuf cmp_off, cmp_stage;  // offsets and compacted cells of the rows on the device
    int64_t last_d2h = 0;      // bytes the last walk call copied device to host
    std::chrono::steady_clock::time_point walk_t0;  // start of the running walk call (host clock)
    int host_link_pct = 62;    // percent of host-output rows copied whole (the rest expanded on the host)
    int host_threads = 0;      // host threads expanding those rows (0: the CPUs the process may use, <= 32)
    int evict_mode = 0;        // node view eviction: 0 chooses, 1 counts evicted endpoints, 2 per-node search
    int32_t mirror_min = 1 << 20;  // live entries from which a node copies its range ahead of a slide

    // Temporal Node2Vec: return / in-out parameters; the live-pair table kept
    // by ingest once q != 1 (pt_cap slots, a power of two; pt_ub bounds the
    // used slots)
    double n2v_p = 1.0, n2v_q = 1.0;
    bool pt_on = false;
    tw::DBuf pt;
    int64_t pt_cap = 0, pt_ub = 0;

    // backward walks of directed graphs: a handle over the reversed edges
    // (dst, src, ts), fed every batch; its node view is the in-view
    tempest *rev = nullptr;
    tempest_walk_stats last_ws{};
    cudaEvent_t kev[2] = {nullptr, nullptr};  // brackets the walk kernels of the last call
    bool kev_valid = false;
    cudaEvent_t eev[2] = {nullptr, nullptr};  // brackets the node view's eviction of the last batch
    bool eev_valid = false;
    int64_t pending_launches = 0;
    std::string err;
};

namespace tw {

// A named NVTX range on the calling host thread for the lifetime of the
// object: the stages of an ingest and of a walk call show up by name in a
// timeline profiler (NVTX is header-only; without a tool attached a range
// costs a branch).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Consecutive stages of one function: next() closes the open range and
// opens the next; the last one closes with the object.
struct NvtxStages {
    bool open = false;
    void next(const char *name)
    {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~NvtxStages()
    {
        if (open) nvtxRangePop();
    }
};

// allocation helpers (capi.cu)
int ensure(tempest_t *h, DBuf &b, size_t bytes, bool headroom = false);
void release(tempest_t *h, DBuf &b);
int fail(tempest_t *h, int code, const char *fmt, ...);
int cuda_check(tempest_t *h, cudaError_t e, const char *what);
bool is_device_ptr(const void *p);

// ingest.cu
// The handle's counters before an ingest.  Through one ingest the store's
// previous live range stays in place (an append writes past it, a move or a
// merge writes the other buffer), so restoring these counters and rebuilding
// the views from the store undoes the ingest.
struct IngestUndo {
    int64_t m, G, N, M, Gn, dropped, evicted, seq_next, cutoff;
    int64_t s_lo, s_hi, s_cap, s_base, tg_lo, tg_hi, n_act, S;
    int has_cutoff, cur;
};
// Ingests one batch; on an error after the store changed (a failed
// allocation, a failed consistency check) the state is restored first, so
// a failed call leaves the handle as it was.  undo (nullable) receives the
// state before a successful call, for ingest_undo.
int ingest_batch(tempest_t *h, const int32_t *src, const int32_t *dst, const int64_t *ts, int64_t n,
                 tempest_ingest_stats *stats, IngestUndo *undo = nullptr);
// Restores the state recorded before the handle's last ingest (no other
// ingest since) and marks the views for a rebuild.
void ingest_undo(tempest_t *h, const IngestUndo &u);
// Rebuilds the views and the pair table from the store when an undo left them
// stale (no-op otherwise).  Every call that reads a view runs it first.
int views_repair(tempest_t *h);

// nodeview.cu
int nv_ensure_nodes(tempest_t *h, int64_t N);
int nv_build(tempest_t *h);
int nv_append(tempest_t *h, const int32_t *ev_src, const int32_t *ev_dst, int64_t n_ev, int64_t new_lo, int64_t nbk,
              int64_t N_old);
// the append's bookkeeping once its counters (h->nvc) were read back into hc;
// *rebuild when a pool could not serve a region (nothing was applied)
int nv_append_finish(tempest_t *h, const NvCounters *hc, bool *rebuild);
// allocates what nv_append will need for the batch, before anything changes
int nv_prepare_append(tempest_t *h, int64_t n_ev, int64_t nbk, int64_t N_old, int64_t N_new);
// canonical NODE_OFF / NODE_ORDER / NODE_GROUP_OFF / NODE_GIDX into device memory
int nv_export(tempest_t *h, int which, int32_t *out);
// timestamp-group starts relative to the live head, plus m (G + 1 values)
int ts_export(tempest_t *h, int32_t *out);

// pairs.cu
int pt_rebuild(tempest_t *h, unsigned long long *status);
int pt_update(tempest_t *h, const int32_t *ev_src, const int32_t *ev_dst, int64_t n_ev, int64_t add_lo,
              int64_t n_add, unsigned long long *status);

// walks.cu
struct WalkRequest;
// the handle whose index a walk of the given direction reads (h itself for
// forward walks and undirected graphs); null when backward walks are off
tempest_t *view_handle(tempest_t *h, int direction);
struct WalkRequest {
    int64_t n_walks;
    int32_t cap;               // row stride
    int32_t max_len;           // when len_arr == nullptr
    const int32_t *len_arr;    // device, nullable
    int bias;                  // when bias_arr == nullptr
    const uint8_t *bias_arr;   // device, nullable
    int start_policy;
    int64_t pn_k;              // PER_NODE: walks per active node
    uint64_t seed;
    int32_t *node;             // device
    int64_t *ts;               // device
    int32_t *len;              // device
    int want_w = 0;            // per-walk biases known to include the weight-based one
    int direction = 0;         // 1: backward walks
    int may_n2v = 1;           // per-walk biases may include Node2Vec (host arrays are scanned)
    int no_pad = 0;            // the lane walker may leave the cells after each walk unwritten
};
int walks_run(tempest_t *h, const WalkRequest &rq);
// pads rows [0, n) of a walk output after their lengths (node -1, ts
// INT64_MIN), one streaming pass on the handle's stream
void pad_rows(tempest_t *h, int64_t n, int32_t cap, const int32_t *len, int32_t *node, int64_t *ts);
// builds the time-bucket tables of the live state on the handle's stream
// (no-op when they are current); every walk form calls it before launching
int prepare_walk_index(tempest_t *h);
// lists the active nodes of the live state in id order (no-op when current)
int prepare_active_nodes(tempest_t *h);
// group weights and their suffix sums for weight-based walks (weights.cu)
int prepare_weights(tempest_t *h);
// weights of the groups an append created or grew (weights.cu); runs after
// the node view scatter of the batch
int nv_append_weights(tempest_t *h, int64_t nbe);
// walks per active node of a PER_NODE request (capi.cu)
int per_node_k(tempest_t *h, int start_policy, int64_t n_walks, int64_t &k, const char *who);
int sample_index_run(tempest_t *h, const uint64_t *ub, const int64_t *n, int64_t count, int bias, double lambda,
                     int64_t *out);

}  // namespace tw
