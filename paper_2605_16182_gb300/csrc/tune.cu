// tune.cu -- tuning knobs of the walk forms and the autotuner that picks
// them by timing walk calls on the live index (the degree thresholds and the
// mega-hub split of Sec. 2.4.3-2.4.5, the density of the hop search index,
// the persistent walker's CTAs per SM, and the walk form itself).
//
// Every knob changes only the mapping of work to threads, never a draw (all
// randomness is keyed by (seed, walk, hop)), so the tuner only measures.
#include <algorithm>

#include "engine.cuh"

using namespace tw;

namespace {

struct Cfg {
    int sched, bkt_log, w_warp, mega, ctas, pad_pass;
};

Cfg current(const tempest_t *h)
{
    return Cfg{h->sched, h->bkt_log, h->coop_w_warp, h->coop_mega, h->stream_ctas, h->pad_pass};
}

void apply(tempest_t *h, const Cfg &c)
{
    h->sched = c.sched;
    if (h->bkt_log != c.bkt_log) {
        h->bkt_log = c.bkt_log;
        h->bkt_ver = -1;  // rebuild the bucket tables at the new density
    }
    h->coop_w_warp = c.w_warp;
    h->coop_mega = c.mega;
    h->stream_ctas = c.ctas;
    h->pad_pass = c.pad_pass;
}

struct Tuner {
    tempest_t *h;
    WalkRequest rq;
    bool per_ingest = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tempest_tune_report rep{};

    // Minimum call time of 3 timed calls after one warm-up; < 0 on error.
    int time_cfg(const Cfg &c, double &ms)
    {
        apply(h, c);
        int rc;
        if ((rc = prepare_walk_index(h))) return rc;
        if ((rc = walks_run(h, rq))) return rc;
        double best = 1e300;
        for (int r = 0; r < 3; r++) {
            if (per_ingest) h->state_ver++;  // as after an ingest: the call rebuilds the derived indexes
            cudaEventRecord(e0, h->stream);
            if ((rc = walks_run(h, rq))) return rc;
            cudaEventRecord(e1, h->stream);
            if ((rc = cuda_check(h, cudaEventSynchronize(e1), "autotune"))) return rc;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, (double)t);
        }
        ms = best;
        if (rep.n_trials < TEMPEST_TUNE_MAX_TRIALS) {
            tempest_tune_trial &tr = rep.trials[rep.n_trials++];
            tr.sched = c.sched;
            tr.bkt_log = c.bkt_log;
            tr.coop_w_warp = c.w_warp;
            tr.coop_mega = c.mega;
            tr.stream_ctas = c.ctas;
            tr.pad_pass = c.pad_pass;
            tr.ms = best;
        }
        return TEMPEST_OK;
    }

    // Tries each value of one knob from the best configuration so far.
    template <class Set>
    int sweep(Cfg &best, double &best_ms, const int *vals, int n, Set set)
    {
        for (int i = 0; i < n; i++) {
            Cfg c = best;
            set(c, vals[i]);
            if (c.sched == best.sched && c.bkt_log == best.bkt_log && c.w_warp == best.w_warp &&
                c.mega == best.mega && c.ctas == best.ctas && c.pad_pass == best.pad_pass)
                continue;
            double ms;
            int rc = time_cfg(c, ms);
            if (rc) return rc;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        return TEMPEST_OK;
    }
};

}  // namespace

extern "C" {

int tempest_set_tuning(tempest_t *h, int knob, int64_t value)
{
    if (!h) return TEMPEST_EINVAL;
    switch (knob) {
        case TEMPEST_TUNE_BKT_LOG:
            if (value < 0 || value > 5) return fail(h, TEMPEST_EINVAL, "tuning: bucket log %lld outside [0, 5]",
                                                    (long long)value);
            if (h->bkt_log != (int)value) {
                h->bkt_log = (int)value;
                h->bkt_ver = -1;
            }
            return TEMPEST_OK;
        case TEMPEST_TUNE_COOP_W_WARP:
            if (value < 1 || value > 256) return fail(h, TEMPEST_EINVAL, "tuning: W_warp %lld outside [1, 256]",
                                                      (long long)value);
            h->coop_w_warp = (int)value;
            return TEMPEST_OK;
        case TEMPEST_TUNE_COOP_MEGA:
            if (value < 256 || value > (1ll << 30))
                return fail(h, TEMPEST_EINVAL, "tuning: mega-hub split %lld outside [256, 2^30]", (long long)value);
            h->coop_mega = (int)value;
            return TEMPEST_OK;
        case TEMPEST_TUNE_STREAM_CTAS:
            if (value < 0 || value > 16) return fail(h, TEMPEST_EINVAL, "tuning: CTAs per SM %lld outside [0, 16]",
                                                     (long long)value);
            h->stream_ctas = (int)value;
            return TEMPEST_OK;
        case TEMPEST_TUNE_PAD_PASS:
            if (value < 0 || value > 1) return fail(h, TEMPEST_EINVAL, "tuning: padding pass %lld is not 0 or 1",
                                                    (long long)value);
            h->pad_pass = (int)value;
            return TEMPEST_OK;
        case TEMPEST_TUNE_HOST_LINK_PCT:
            if (value < 0 || value > 100) return fail(h, TEMPEST_EINVAL, "tuning: host link share %lld outside [0, 100]",
                                                      (long long)value);
            h->host_link_pct = (int)value;
            return TEMPEST_OK;
        case TEMPEST_TUNE_HOST_THREADS:
            if (value < 0 || value > 256) return fail(h, TEMPEST_EINVAL, "tuning: host threads %lld outside [0, 256]",
                                                      (long long)value);
            h->host_threads = (int)value;
            return TEMPEST_OK;
        case TEMPEST_TUNE_EVICT:
            if (value < 0 || value > 2) return fail(h, TEMPEST_EINVAL, "tuning: eviction mode %lld is not 0, 1 or 2",
                                                    (long long)value);
            h->evict_mode = (int)value;
            return TEMPEST_OK;
        case TEMPEST_TUNE_MIRROR_MIN:
            if (value < 16 || value > (1 << 30))
                return fail(h, TEMPEST_EINVAL, "tuning: copy-ahead threshold %lld outside [16, 2^30]", (long long)value);
            h->mirror_min = (int32_t)value;
            return TEMPEST_OK;
        default:
            return fail(h, TEMPEST_EINVAL, "tuning: unknown knob %d", knob);
    }
}

int tempest_get_tuning(tempest_t *h, int knob, int64_t *value)
{
    if (!h || !value) return TEMPEST_EINVAL;
    switch (knob) {
        case TEMPEST_TUNE_BKT_LOG: *value = h->bkt_log; return TEMPEST_OK;
        case TEMPEST_TUNE_COOP_W_WARP: *value = h->coop_w_warp; return TEMPEST_OK;
        case TEMPEST_TUNE_COOP_MEGA: *value = h->coop_mega; return TEMPEST_OK;
        case TEMPEST_TUNE_STREAM_CTAS: *value = h->stream_ctas; return TEMPEST_OK;
        case TEMPEST_TUNE_PAD_PASS: *value = h->pad_pass; return TEMPEST_OK;
        case TEMPEST_TUNE_HOST_LINK_PCT: *value = h->host_link_pct; return TEMPEST_OK;
        case TEMPEST_TUNE_HOST_THREADS: *value = h->host_threads; return TEMPEST_OK;
        case TEMPEST_TUNE_EVICT: *value = h->evict_mode; return TEMPEST_OK;
        case TEMPEST_TUNE_MIRROR_MIN: *value = h->mirror_min; return TEMPEST_OK;
        default: return fail(h, TEMPEST_EINVAL, "tuning: unknown knob %d", knob);
    }
}

static int autotune_impl(tempest_t *h, int64_t n_walks, int32_t max_len, const int32_t *len_arr, int bias,
                         const uint8_t *bias_arr, int start_policy, uint64_t seed, int32_t flags,
                         tempest_tune_report *out);

int tempest_autotune(tempest_t *h, int64_t n_walks, int32_t max_len, int bias, int start_policy, uint64_t seed,
                     int32_t flags, tempest_tune_report *out)
{
    if (!h) return TEMPEST_EINVAL;
    if (bias < 0 || bias > 4) return fail(h, TEMPEST_EINVAL, "tempest_autotune: unknown bias %d", bias);
    return autotune_impl(h, n_walks, max_len, nullptr, bias, nullptr, start_policy, seed, flags, out);
}

int tempest_autotune_mixed(tempest_t *h, int64_t n_walks, const int32_t *max_len_arr, int32_t max_len_cap,
                           const uint8_t *bias_arr, int start_policy, uint64_t seed, int32_t flags,
                           tempest_tune_report *out)
{
    if (!h) return TEMPEST_EINVAL;
    if (!max_len_arr || !bias_arr || !is_device_ptr(max_len_arr) || !is_device_ptr(bias_arr))
        return fail(h, TEMPEST_EINVAL, "tempest_autotune_mixed: per-walk arrays must be device memory");
    return autotune_impl(h, n_walks, max_len_cap, max_len_arr, 0, bias_arr, start_policy, seed, flags, out);
}

}  // extern "C"

static int autotune_impl(tempest_t *h, int64_t n_walks, int32_t max_len, const int32_t *len_arr, int bias,
                         const uint8_t *bias_arr, int start_policy, uint64_t seed, int32_t flags,
                         tempest_tune_report *out)
{
    if (n_walks < 1 || max_len < 2 ||
        (start_policy != TEMPEST_START_UNIFORM_EDGE && start_policy != TEMPEST_START_BIASED_TS))
        return fail(h, TEMPEST_EINVAL, "tempest_autotune: bad n_walks, max_len or start policy");
    if ((flags & ~(TEMPEST_TUNE_FORMS | TEMPEST_TUNE_PER_INGEST)) != 0)
        return fail(h, TEMPEST_EINVAL, "tempest_autotune: unknown flags");
    if (n_walks > (int64_t)INT32_MAX / 2) return fail(h, TEMPEST_EINVAL, "tempest_autotune: n_walks too large");
    int rc;
    const size_t cells = (size_t)n_walks * (size_t)max_len;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    if ((rc = ensure(h, h->tune_out, up(cells * 8) + up(cells * 4) + up((size_t)n_walks * 4)))) return rc;
    char *base = h->tune_out.as<char>();

    Tuner T;
    T.h = h;
    T.per_ingest = (flags & TEMPEST_TUNE_PER_INGEST) != 0;
    T.rq.n_walks = n_walks;
    T.rq.cap = max_len;
    T.rq.max_len = max_len;
    T.rq.len_arr = len_arr;
    T.rq.bias = bias;
    T.rq.bias_arr = bias_arr;
    T.rq.start_policy = start_policy;
    T.rq.seed = seed;
    T.rq.ts = reinterpret_cast<int64_t *>(base);
    T.rq.node = reinterpret_cast<int32_t *>(base + up(cells * 8));
    T.rq.len = reinterpret_cast<int32_t *>(base + up(cells * 8) + up(cells * 4));
    cudaEventCreate(&T.e0);
    cudaEventCreate(&T.e1);

    const Cfg start = current(h);
    Cfg best = start;
    double best_ms = 0.0;
    rc = T.time_cfg(best, best_ms);
    const double start_ms = best_ms;
    if (!rc && (flags & TEMPEST_TUNE_FORMS)) {
        const int forms[] = {TEMPEST_SCHED_STREAM, TEMPEST_SCHED_LANE, TEMPEST_SCHED_FULL_WALK, TEMPEST_SCHED_COOP,
                             TEMPEST_SCHED_GRAPH};
        rc = T.sweep(best, best_ms, forms, 5, [](Cfg &c, int v) { c.sched = v; });
    }
    if (!rc) {
        const int logs[] = {0, 1, 2, 3, 4};
        rc = T.sweep(best, best_ms, logs, 5, [](Cfg &c, int v) { c.bkt_log = v; });
    }
    if (!rc && (best.sched == TEMPEST_SCHED_STREAM || best.sched == TEMPEST_SCHED_LANE)) {
        const int ctas[] = {2, 3, 4, 5, 6};
        rc = T.sweep(best, best_ms, ctas, 5, [](Cfg &c, int v) { c.ctas = v; });
    }
    if (!rc && best.sched == TEMPEST_SCHED_LANE && !T.rq.len_arr) {
        const int pp[] = {0, 1};
        rc = T.sweep(best, best_ms, pp, 2, [](Cfg &c, int v) { c.pad_pass = v; });
    }
    if (!rc && best.sched == TEMPEST_SCHED_COOP) {
        const int ww[] = {1, 2, 4, 8, 16, 32};
        rc = T.sweep(best, best_ms, ww, 6, [](Cfg &c, int v) { c.w_warp = v; });
        const int mg[] = {1024, 2048, 4096, 8192, 16384, 65536};
        if (!rc) rc = T.sweep(best, best_ms, mg, 6, [](Cfg &c, int v) { c.mega = v; });
    }
    cudaEventDestroy(T.e0);
    cudaEventDestroy(T.e1);
    apply(h, rc ? start : best);
    if (rc) return rc;
    if ((rc = prepare_walk_index(h))) return rc;
    if (out) {
        T.rep.sched = best.sched;
        T.rep.bkt_log = best.bkt_log;
        T.rep.coop_w_warp = best.w_warp;
        T.rep.coop_mega = best.mega;
        T.rep.stream_ctas = best.ctas;
        T.rep.pad_pass = best.pad_pass;
        T.rep.best_ms = best_ms;
        T.rep.start_ms = start_ms;
        *out = T.rep;
    }
    return TEMPEST_OK;
}
