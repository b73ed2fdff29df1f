/*
 * Tempest CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of what the streaming temporal
 * random-walk engine computes (Salehin, Parisis, Berthouze, "Tempest: A
 * GPU-Accelerated Engine for Streaming Temporal Random Walks").  It exists to
 * check the CUDA library; only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no code,
 * header, table or helper with the CUDA library and must never be used as a
 * fallback for it.
 *
 * Every step follows the paper's definitions directly, with no blocking,
 * fusion or reordering:
 *   - temporal graph, forward neighbourhood Gamma_t(v) = {(v,w,t') : t' > t},
 *     ties on timestamps broken uniformly                        (Sec. 2.1)
 *   - dual index: one edge store, a timestamp-grouped view and a node-and-
 *     timestamp-grouped view, both offset arrays over the store   (Sec. 2.3)
 *   - index-based closed-form samplers, Eq. 1 (uniform), Eq. 2 (linear),
 *     Eq. 3 (exponential, replaced by its exact inverse CDF, see below)
 *                                                                 (Sec. 2.5)
 *   - sliding window W(t) = {e : t - Delta <= t_e <= t}, each batch sorted by
 *     timestamp, late edges dropped without retraction            (Sec. 2.6)
 *
 * Readings taken where the paper is silent or garbled:
 *   - seq: every edge passed to ingest gets a global arrival index (dropped
 *     edges too); the store is ordered by (ts, seq), so equal timestamps keep
 *     arrival order.
 *   - window > 0 is the duration Delta with t = max timestamp ingested so far
 *     (window inclusive); window < 0 keeps the -window newest edges, cut at the
 *     timestamp of the (-window)-th newest edge, keeping that whole timestamp
 *     group; window == 0 keeps everything.
 *   - late edge: ts < the cut-off in force before the batch; dropped, counted.
 *   - node ids are int32 >= 0; the node arrays span [0, 1 + max id seen].
 *   - undirected graphs index every edge under both endpoints (slot 2p for the
 *     source side, 2p+1 for the destination side of store position p).
 *   - uniform bias draws over edges of Gamma_t(v); linear / exponential bias
 *     draw a timestamp group (the ordinal index i of Sec. 2.5) and then an
 *     edge uniformly inside the group.
 *   - Eq. 3 as printed cannot return index n-1; the oracle uses the exact
 *     inverse CDF of weights exp(lambda*i), i in [0,n):
 *       x = n + log(u + (1-u) exp(-lambda n)) / lambda.
 *   - RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = seed,
 *     counter = (hop, 0, walk_lo, walk_hi); two 53-bit uniforms per block.
 *   - max_len counts nodes; the start edge contributes two nodes.
 *
 * Build with -ffp-contract=off: the linear and exponential samplers are
 * evaluated left to right in IEEE double with no fused multiply-add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

#define BIAS_UNIFORM 0
#define BIAS_LINEAR 1
#define BIAS_EXP 2
#define BIAS_EXP_WEIGHT 3
#define BIAS_NODE2VEC 4

/* Temporal Node2Vec: proposals drawn per hop before the walk ends */
#define N2V_MAX_TRIALS 4096

#define START_UNIFORM_EDGE 0
#define START_BIASED_TS 1
#define START_PER_NODE 2

typedef struct {
    int32_t src, dst;
    int64_t ts;
    int64_t seq;
} orc_edge;

typedef struct {
    int64_t node; /* the node under which the entry is indexed */
    int64_t slot; /* store position (directed) or 2*position + side */
} orc_entry;

typedef struct orc {
    int64_t window;
    int directed;
    double lambda_hop;   /* exponential rate per timestamp group for hops */
    double lambda_start; /* > 0: fixed rate for start selection; 0: 1/G_tot */
    double lambda_w;     /* weight-based sampler: rate per timestamp unit */
    double n2v_p, n2v_q; /* Temporal Node2Vec return / in-out parameters */

    orc_edge *live; /* live edges in (ts, seq) order */
    int64_t m;
    int64_t seq_next;
    int has_cutoff;
    int64_t cutoff;
    int64_t n_nodes; /* 1 + max id seen */
    int64_t dropped_late, evicted;

    /* timestamp-grouped view */
    int64_t *ts_group_off; /* G_tot + 1 */
    int64_t G_tot;
    /* node-and-timestamp-grouped view */
    int64_t *node_off;       /* n_nodes + 1 */
    int64_t *node_order;     /* M slots */
    int64_t M;
    int64_t *node_group_off; /* Gn + 1, absolute positions in node_order */
    int64_t *node_gidx;      /* n_nodes + 1, first group index of node v */
    int64_t Gn;
} orc;

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the SC'11 paper's definition.                  */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The random block a walk uses at a hop (hop 0 = start selection); word 1
 * of the counter numbers the draws of one hop (0 for every sampler but the
 * Node2Vec rejection loop). */
static void draw_block(uint64_t seed, uint64_t walk, uint32_t hop, uint32_t word1, uint32_t r[4])
{
    uint32_t ctr[4] = {hop, word1, (uint32_t)walk, (uint32_t)(walk >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, r);
}

static void walk_block(uint64_t seed, uint64_t walk, uint32_t hop, uint32_t r[4])
{
    draw_block(seed, walk, hop, 0u, r);
}

/* 53-bit uniform in [0, 1) from two 32-bit words. */
double orc_u53(uint32_t hi, uint32_t lo)
{
    uint64_t b = (((uint64_t)hi << 32) | lo) >> 11;
    return (double)b * (1.0 / 9007199254740992.0); /* 2^-53 */
}

/* ------------------------------------------------------------------ */
/* Index-based samplers (Sec. 2.5).  Returns x (the continuous inverse */
/* CDF value); the drawn index is clamp(floor(x), 0, n-1).            */
/* ------------------------------------------------------------------ */
double orc_sampler_x(double u, int64_t n, int bias, double lambda)
{
    double nd = (double)n;
    if (bias == BIAS_UNIFORM) {
        /* Eq. 1 */
        return u * nd;
    }
    if (bias == BIAS_LINEAR) {
        /* Eq. 2: weight i+1 on index i */
        double t = 4.0 * u;
        t = t * nd;
        t = t * (nd + 1.0);
        t = 1.0 + t;
        return (sqrt(t) - 1.0) * 0.5;
    }
    /* exponential, weight exp(lambda*i) on index i (exact form of Eq. 3) */
    {
        double a = -lambda * nd;
        double e = exp(a);
        double s = u + (1.0 - u) * e;
        return nd + log(s) / lambda;
    }
}

int64_t orc_sampler_index(double u, int64_t n, int bias, double lambda)
{
    double x = orc_sampler_x(u, n, bias, lambda);
    if (!(x >= 0.0)) return 0; /* NaN, -inf or negative */
    double f = floor(x);
    if (f >= (double)(n - 1)) return n - 1;
    return (int64_t)f;
}

/*
 * Error bound of the double evaluation of orc_sampler_x, in units of x: the
 * largest |x_fl - x| that rounding can cause, by first-order analysis with
 * unit roundoff eps = 2^-53 per IEEE operation and exp / log within one ulp
 * (2 eps relative), the accuracy glibc and CUDA state for them.  Two
 * evaluations of the same formula (this one and the GPU's) can floor to
 * different indexes only where x lies within twice this bound of an integer.
 *   uniform (Eq. 1): one rounded product, eps x.
 *   linear (Eq. 2): 4 u n (n + 1) + 1 rounded four times, the square root
 *     and the last two steps once each: within 4 eps (x + 1).
 *   exponential (exact form of Eq. 3), y = x - n = log(s) / lambda:
 *     a = fl(lambda n) errs by eps lambda n, so exp(a) carries
 *     eps (lambda n + 2) relative; 1 - u is exact for u = k 2^-53; the
 *     product and the sum give s a relative error of at most
 *     eps (1 + m (3 + lambda n)), m = (1 - u) e / s <= 1; log adds
 *     2 eps |lambda y| (that is 2 eps |y| after the division), the division
 *     eps |y| and the final sum eps |x|:
 *       |x_fl - x| <= eps (|x| + 3 |y| + (1 + m (3 + lambda n)) / lambda).
 *   Every coefficient is doubled below to cover the second-order terms.
 */
double orc_sampler_x_bound(double u, int64_t n, int bias, double lambda)
{
    const double eps = 1.0 / 9007199254740992.0; /* 2^-53 */
    const double nd = (double)n;
    const double x = orc_sampler_x(u, n, bias, lambda);
    const double ax = x == x ? fabs(x) : 0.0;
    if (bias == BIAS_UNIFORM) return 2.0 * eps * ax;
    if (bias == BIAS_LINEAR) return 8.0 * eps * (ax + 1.0);
    const double e = exp(-lambda * nd);
    const double s = u + (1.0 - u) * e;
    const double m = s > 0.0 ? (1.0 - u) * e / s : 1.0;
    const double ay = x == x ? fabs(x - nd) : 0.0;
    return eps * (2.0 * ax + 6.0 * ay + (2.0 + m * (6.0 + 2.0 * lambda * nd)) / lambda);
}

/* Distance of x to the nearest integer in units of the bound b (0 for NaN). */
static double bound_margin(double x, double b)
{
    if (!(x == x)) return 0.0;
    double r = x - floor(x + 0.5);
    if (r < 0) r = -r;
    return r / (b > 0.0 ? b : 4.9406564584124654e-324);
}

/* Many draws: u = k[i] * 2^-53.  out[i] = index; margin[i] (nullable) =
 * |x - nearest integer| in units of orc_sampler_x_bound. */
void orc_sampler_batch(const uint64_t *k, const int64_t *n, int64_t count, int bias, double lambda,
                       int64_t *out, double *margin)
{
    for (int64_t i = 0; i < count; i++) {
        double u = (double)(k[i] & ((1ull << 53) - 1)) * (1.0 / 9007199254740992.0);
        out[i] = orc_sampler_index(u, n[i], bias, lambda);
        if (margin)
            margin[i] = bound_margin(orc_sampler_x(u, n[i], bias, lambda),
                                     orc_sampler_x_bound(u, n[i], bias, lambda));
    }
}

/* uniform index in [0, n) from u (Eq. 1 with the clamp) */
static int64_t uniform_index(double u, int64_t n)
{
    return orc_sampler_index(u, n, BIAS_UNIFORM, 1.0);
}

/* ------------------------------------------------------------------ */
/* Handle                                                             */
/* ------------------------------------------------------------------ */
orc *orc_create(int64_t window, int directed)
{
    orc *o = (orc *)calloc(1, sizeof(orc));
    if (!o) return NULL;
    o->window = window;
    o->directed = directed ? 1 : 0;
    o->lambda_hop = 1.0;
    o->lambda_start = 0.0;
    o->lambda_w = 1e-9;
    o->n2v_p = 1.0;
    o->n2v_q = 1.0;
    o->ts_group_off = (int64_t *)calloc(1, sizeof(int64_t));
    o->node_off = (int64_t *)calloc(1, sizeof(int64_t));
    o->node_gidx = (int64_t *)calloc(1, sizeof(int64_t));
    o->node_group_off = (int64_t *)calloc(1, sizeof(int64_t));
    return o;
}

void orc_destroy(orc *o)
{
    if (!o) return;
    free(o->live);
    free(o->ts_group_off);
    free(o->node_off);
    free(o->node_order);
    free(o->node_group_off);
    free(o->node_gidx);
    free(o);
}

int orc_set_weight_rate(orc *o, double lambda_w)
{
    if (!(lambda_w > 0.0)) return ORC_EINVAL;
    o->lambda_w = lambda_w;
    return ORC_OK;
}

/*
 * The weight-based exponential sampler of Sec. 2.5 over n timestamp groups
 * (ascending timestamps ts[0..n), sizes size[0..n)): every edge weighs
 * exp(lambda (t_e - t_min)) with t_min = ts[0], the earliest timestamp of
 * the neighbourhood; r = u * (total weight); the result is the group holding
 * the first edge whose running sum reaches r (edges of one group weigh the
 * same, so the group follows from the group sums).  Every weight is
 * multiplied by exp(-lambda (t_max - t_min)), a common factor that cancels
 * from r and the running sum: the weights become exp(lambda (t_e - t_max))
 * <= 1, which stays finite where the raw form overflows (lambda (t_max -
 * t_min) > 709).  margin (nullable) receives the distance of r to the
 * nearer boundary of that group's interval, relative to the total.
 */
int64_t orc_weight_pick(const int64_t *ts, const int64_t *size, int64_t n, double lambda, double u, double *margin)
{
    const int64_t tmax = ts[n - 1];
    double total = 0.0;
    for (int64_t g = 0; g < n; g++) total += (double)size[g] * exp(lambda * (double)(ts[g] - tmax));
    const double r = u * total;
    double run = 0.0;
    for (int64_t g = 0; g < n; g++) {
        const double before = run;
        run += (double)size[g] * exp(lambda * (double)(ts[g] - tmax));
        if (run >= r || g == n - 1) {
            if (margin) {
                double a = r - before, b = run - r;
                if (a < 0) a = -a;
                if (b < 0) b = -b;
                *margin = (a < b ? a : b) / total;
            }
            return g;
        }
    }
    return n - 1;
}

int orc_set_node2vec(orc *o, double p, double q)
{
    if (!(p >= 1e-3 && p <= 1e3) || !(q >= 1e-3 && q <= 1e3)) return ORC_EINVAL;
    o->n2v_p = p;
    o->n2v_q = q;
    return ORC_OK;
}

int orc_set_bias_params(orc *o, double lambda_hop, double lambda_start)
{
    if (!(lambda_hop > 0.0) || !(lambda_start >= 0.0)) return ORC_EINVAL;
    o->lambda_hop = lambda_hop;
    o->lambda_start = lambda_start;
    return ORC_OK;
}

static int cmp_edge_ts_seq(const void *a, const void *b)
{
    const orc_edge *x = (const orc_edge *)a, *y = (const orc_edge *)b;
    if (x->ts != y->ts) return x->ts < y->ts ? -1 : 1;
    if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
    return 0;
}

static int cmp_entry(const void *a, const void *b)
{
    const orc_entry *x = (const orc_entry *)a, *y = (const orc_entry *)b;
    if (x->node != y->node) return x->node < y->node ? -1 : 1;
    if (x->slot != y->slot) return x->slot < y->slot ? -1 : 1;
    return 0;
}

static int64_t slot_ts(const orc *o, int64_t slot)
{
    int64_t pos = o->directed ? slot : (slot >> 1);
    return o->live[pos].ts;
}

/* the endpoint reached by traversing the entry */
static int32_t slot_other(const orc *o, int64_t slot)
{
    if (o->directed) return o->live[slot].dst;
    int64_t pos = slot >> 1;
    return (slot & 1) ? o->live[pos].src : o->live[pos].dst;
}

/* Rebuild both views from scratch over the live store (Sec. 2.3). */
static int rebuild_views(orc *o)
{
    int64_t m = o->m, N = o->n_nodes;

    /* timestamp-grouped view: start of each run of equal timestamps */
    free(o->ts_group_off);
    o->ts_group_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!o->ts_group_off) return ORC_ENOMEM;
    int64_t G = 0;
    for (int64_t i = 0; i < m; i++)
        if (i == 0 || o->live[i].ts != o->live[i - 1].ts) o->ts_group_off[G++] = i;
    o->ts_group_off[G] = m;
    o->G_tot = G;

    /* node-and-timestamp-grouped view: entries ordered by (node, slot) */
    int64_t M = o->directed ? m : 2 * m;
    orc_entry *ent = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(M > 0 ? M : 1));
    if (!ent) return ORC_ENOMEM;
    for (int64_t p = 0; p < m; p++) {
        if (o->directed) {
            ent[p].node = o->live[p].src;
            ent[p].slot = p;
        } else {
            ent[2 * p].node = o->live[p].src;
            ent[2 * p].slot = 2 * p;
            ent[2 * p + 1].node = o->live[p].dst;
            ent[2 * p + 1].slot = 2 * p + 1;
        }
    }
    qsort(ent, (size_t)M, sizeof(orc_entry), cmp_entry);

    free(o->node_order);
    o->node_order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1));
    free(o->node_off);
    o->node_off = (int64_t *)calloc((size_t)(N + 1), sizeof(int64_t));
    if (!o->node_order || !o->node_off) { free(ent); return ORC_ENOMEM; }
    for (int64_t i = 0; i < M; i++) {
        o->node_order[i] = ent[i].slot;
        o->node_off[ent[i].node + 1] += 1; /* count, turned into offsets below */
    }
    for (int64_t v = 0; v < N; v++) o->node_off[v + 1] += o->node_off[v];

    /* timestamp sub-groups inside each node's segment */
    free(o->node_group_off);
    free(o->node_gidx);
    o->node_group_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
    o->node_gidx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (!o->node_group_off || !o->node_gidx) { free(ent); return ORC_ENOMEM; }
    int64_t Gn = 0;
    for (int64_t v = 0; v < N; v++) {
        o->node_gidx[v] = Gn;
        for (int64_t i = o->node_off[v]; i < o->node_off[v + 1]; i++) {
            if (i == o->node_off[v] ||
                slot_ts(o, o->node_order[i]) != slot_ts(o, o->node_order[i - 1]))
                o->node_group_off[Gn++] = i;
        }
    }
    o->node_gidx[N] = Gn;
    o->node_group_off[Gn] = M;
    o->Gn = Gn;
    o->M = M;
    free(ent);
    return ORC_OK;
}

/* Ingest one batch (Sec. 2.6). */
int orc_ingest(orc *o, const int32_t *src, const int32_t *dst, const int64_t *ts, int64_t n)
{
    if (n < 0) return ORC_EINVAL;
    if (n > 0 && (!src || !dst || !ts)) return ORC_EINVAL;
    for (int64_t i = 0; i < n; i++)
        if (src[i] < 0 || dst[i] < 0 || ts[i] == INT64_MIN || ts[i] == INT64_MAX) return ORC_EINVAL;

    /* 1. arrival index for every edge; drop late edges */
    orc_edge *batch = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)(n > 0 ? n : 1));
    if (!batch) return ORC_ENOMEM;
    int64_t b = 0;
    for (int64_t i = 0; i < n; i++) {
        if (src[i] + 1 > o->n_nodes) o->n_nodes = (int64_t)src[i] + 1;
        if (dst[i] + 1 > o->n_nodes) o->n_nodes = (int64_t)dst[i] + 1;
        if (o->has_cutoff && ts[i] < o->cutoff) {
            o->dropped_late++;
            continue;
        }
        batch[b].src = src[i];
        batch[b].dst = dst[i];
        batch[b].ts = ts[i];
        batch[b].seq = o->seq_next + i;
        b++;
    }
    o->seq_next += n;

    /* 2. sort the batch by timestamp (arrival order among ties) */
    qsort(batch, (size_t)b, sizeof(orc_edge), cmp_edge_ts_seq);

    /* 3. merge into the store, keyed by (ts, seq) */
    int64_t mm = o->m + b;
    orc_edge *merged = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)(mm > 0 ? mm : 1));
    if (!merged) { free(batch); return ORC_ENOMEM; }
    {
        int64_t i = 0, j = 0, k = 0;
        while (i < o->m && j < b) {
            if (cmp_edge_ts_seq(&o->live[i], &batch[j]) <= 0) merged[k++] = o->live[i++];
            else merged[k++] = batch[j++];
        }
        while (i < o->m) merged[k++] = o->live[i++];
        while (j < b) merged[k++] = batch[j++];
    }
    free(batch);

    /* 4. advance the window cut-off */
    if (o->window > 0 && mm > 0) {
        int64_t tmax = merged[mm - 1].ts;
        int64_t c;
        if (tmax < INT64_MIN + o->window) c = INT64_MIN;
        else c = tmax - o->window;
        if (!o->has_cutoff || c > o->cutoff) o->cutoff = c;
        o->has_cutoff = 1;
    } else if (o->window < 0) {
        int64_t W = -o->window;
        if (mm > W) {
            int64_t c = merged[mm - W].ts;
            if (!o->has_cutoff || c > o->cutoff) o->cutoff = c;
            o->has_cutoff = 1;
        }
    }

    /* 5. evict the prefix older than the cut-off */
    int64_t first = 0;
    if (o->has_cutoff)
        while (first < mm && merged[first].ts < o->cutoff) first++;
    o->evicted += first;
    free(o->live);
    o->m = mm - first;
    o->live = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)(o->m > 0 ? o->m : 1));
    if (!o->live) { free(merged); return ORC_ENOMEM; }
    memcpy(o->live, merged + first, sizeof(orc_edge) * (size_t)o->m);
    free(merged);

    /* 6. rebuild the dual index */
    return rebuild_views(o);
}

/* First group of node v whose timestamp is > t (upper bound), or g1 when
 * Gamma_t(v) is empty. */
static int64_t first_group_after(const orc *o, int64_t g0, int64_t g1, int64_t t)
{
    int64_t lo = g0, hi = g1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int64_t gts = slot_ts(o, o->node_order[o->node_group_off[mid]]);
        if (gts > t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

/* Margin of a draw with u of n outcomes (see orc_sampler_x_bound). */
static double draw_margin(double u, int64_t n, int bias, double lambda)
{
    return bound_margin(orc_sampler_x(u, n, bias, lambda), orc_sampler_x_bound(u, n, bias, lambda));
}

/* Live (from, to) pairs for the Temporal Node2Vec adjacency test: sorted
 * keys from << 32 | to, both orientations for undirected graphs. */
typedef struct {
    uint64_t *key;
    int64_t n;
} orc_pairs;

static int64_t n2v_pick(const orc *o, const orc_pairs *P, const int64_t *group_off, const int64_t *order, int64_t lo,
                        int64_t hi, int back, int64_t prev, uint64_t seed, uint64_t w, uint32_t h, double *margin,
                        double *bytes);

/*
 * One walk.  Writes up to max_len nodes and timestamps (the first timestamp
 * is INT64_MIN: the start node is reached at no time), returns the length.
 * With START_PER_NODE the walk starts at node `start_node` and its first hop
 * draws from all of that node's live edges (every timestamp is above
 * INT64_MIN); the other policies draw a start edge, which gives two nodes.
 * The hop that appends the node at position p uses Philox counter p - 1.
 * margin (nullable, max_len entries) receives, for each position drawn by a
 * linear or exponential sampler, |x - nearest integer| / max(1, n); other
 * positions receive +inf.  bytes (nullable) accumulates the per-hop sector
 * model of the walk's memory traffic.
 */
static int32_t one_walk(const orc *o, const orc_pairs *P, uint64_t w, int32_t max_len, int bias, int start_policy,
                        int64_t start_node, uint64_t seed, int32_t *node, int64_t *tsout, double *margin,
                        double lambda_start, double *bytes)
{
    for (int32_t i = 0; i < max_len; i++) {
        node[i] = -1;
        tsout[i] = INT64_MIN;
        if (margin) margin[i] = INFINITY;
    }
    if (o->m == 0) return 0;

    uint32_t r[4];
    double u1, u2;
    int32_t len;
    int64_t v, t;
    int64_t prev = -1; /* the node before v (Temporal Node2Vec), none at a PER_NODE start */
    if (start_policy == START_PER_NODE) {
        node[0] = (int32_t)start_node;
        len = 1;
        v = start_node;
        t = INT64_MIN;
    } else {
        walk_block(seed, w, 0, r);
        u1 = orc_u53(r[0], r[1]);
        u2 = orc_u53(r[2], r[3]);
        int64_t k;
        if (start_policy == START_UNIFORM_EDGE) {
            k = uniform_index(u1, o->m);
        } else {
            /* the weight-based and Node2Vec biases start like the index-based exponential */
            const int sb = (bias == BIAS_EXP_WEIGHT || bias == BIAS_NODE2VEC) ? BIAS_EXP : bias;
            int64_t g = orc_sampler_index(u1, o->G_tot, sb, lambda_start);
            if (margin && sb != BIAS_UNIFORM) margin[1] = draw_margin(u1, o->G_tot, sb, lambda_start);
            int64_t a = o->ts_group_off[g], size = o->ts_group_off[g + 1] - a;
            k = a + uniform_index(u2, size);
        }
        int32_t s = o->live[k].src, d = o->live[k].dst;
        if (!o->directed && (r[3] & 1u)) {
            int32_t tmp = s; s = d; d = tmp;
        }
        node[0] = s;
        node[1] = d;
        tsout[1] = o->live[k].ts;
        len = 2;
        if (bytes) *bytes += 3 * 32.0 + 4 + 4 + 8 + 8 + 4;
        prev = s;
        v = d;
        t = o->live[k].ts;
    }

    while (len < max_len) {
        const uint32_t h = (uint32_t)(len - 1);
        int64_t g0 = o->node_gidx[v], g1 = o->node_gidx[v + 1];
        int64_t c = first_group_after(o, g0, g1, t);
        if (c == g1) break; /* Gamma_t(v) is empty */
        walk_block(seed, w, h, r);
        u1 = orc_u53(r[0], r[1]);
        u2 = orc_u53(r[2], r[3]);
        int64_t idx;
        if (bias == BIAS_NODE2VEC) {
            const int64_t slot = n2v_pick(o, P, o->node_group_off, o->node_order, c, g1, 0, prev, seed, w, h,
                                          margin ? &margin[len] : NULL, bytes);
            if (slot < 0) break; /* every proposal rejected */
            node[len] = slot_other(o, slot);
            tsout[len] = slot_ts(o, slot);
            if (bytes) {
                int64_t G = g1 - g0;
                int lg = 0;
                while (((int64_t)1 << lg) < G + 1) lg++;
                int search = lg - 2 > 1 ? lg - 2 : 1;
                *bytes += 32.0 * (1 + search + 1) + 12 + 16;
            }
            prev = v;
            v = node[len];
            t = tsout[len];
            len++;
            continue;
        }
        if (bias == BIAS_UNIFORM) {
            int64_t e0 = o->node_group_off[c], e1 = o->node_off[v + 1];
            idx = e0 + uniform_index(u1, e1 - e0);
        } else if (bias == BIAS_EXP_WEIGHT) {
            const int64_t n = g1 - c;
            int64_t *gts = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
            int64_t *gsz = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
            if (!gts || !gsz) {
                free(gts);
                free(gsz);
                break;
            }
            for (int64_t g = 0; g < n; g++) {
                const int64_t a = o->node_group_off[c + g], b = o->node_group_off[c + g + 1];
                gts[g] = slot_ts(o, o->node_order[a]);
                gsz[g] = b - a;
            }
            double mg = INFINITY;
            const int64_t j = orc_weight_pick(gts, gsz, n, o->lambda_w, u1, &mg);
            free(gts);
            free(gsz);
            /* in units of the rounding either evaluation can make in the
             * running weight: each weight carries about eps (|exponent| + 2)
             * relative (exponents stay within 750 where a weight is not
             * zero), and a running or suffix sum over the node's g1 - g0
             * groups adds eps per group */
            if (margin) margin[len] = mg / ((double)(g1 - g0 + 800) * (1.0 / 9007199254740992.0));
            int64_t e0 = o->node_group_off[c + j], e1 = o->node_group_off[c + j + 1];
            idx = e0 + uniform_index(u2, e1 - e0);
        } else {
            int64_t n = g1 - c;
            int64_t j = orc_sampler_index(u1, n, bias, o->lambda_hop);
            if (margin) margin[len] = draw_margin(u1, n, bias, o->lambda_hop);
            int64_t e0 = o->node_group_off[c + j], e1 = o->node_group_off[c + j + 1];
            idx = e0 + uniform_index(u2, e1 - e0);
        }
        int64_t slot = o->node_order[idx];
        node[len] = slot_other(o, slot);
        tsout[len] = slot_ts(o, slot);
        if (bytes) {
            int64_t G = g1 - g0;
            int lg = 0;
            while (((int64_t)1 << lg) < G + 1) lg++; /* ceil(log2(G+1)) */
            int search = lg - 2 > 1 ? lg - 2 : 1;
            *bytes += 32.0 * (1 + search + 1) + 12 + 16;
        }
        prev = v;
        v = node[len];
        t = tsout[len];
        len++;
    }
    return len;
}

/* Nodes with at least one live entry in the node view, in id order. */
int64_t orc_active_nodes(const orc *o, int32_t *out)
{
    int64_t n = 0;
    for (int64_t v = 0; v < o->n_nodes; v++)
        if (o->node_gidx[v + 1] > o->node_gidx[v]) {
            if (out) out[n] = (int32_t)v;
            n++;
        }
    return n;
}

/* ------------------------------------------------------------------ */
/* Backward walks (Sec. 2.1: "the backward case defined analogously").  */
/* ------------------------------------------------------------------ */
/*
 * Reading: a backward walk on G is a forward walk on the time-reversed graph
 * that holds every live edge (u, v, t) as (v, u, -t), in mirrored arrival
 * order.  So from node v at time t it draws from the in-edges of v earlier
 * than t, Gamma^-_t(v) = {(u, v, t') : t' < t}, taken in the mirrored order
 * (descending timestamp, descending arrival): the samplers' index 0 is the
 * latest such edge or group, and a draw at mirrored position q of a range is
 * the range's element last - q.  Start edges are mirrored the same way
 * (store position m - 1 - k, timestamp group G - 1 - g), and the walk takes
 * the start edge from its destination to its source.
 */
typedef struct {
    int64_t *off, *order, *group_off, *gidx;
    int64_t Gn;
} orc_inview;

static void free_inview(orc_inview *iv)
{
    free(iv->off);
    free(iv->order);
    free(iv->group_off);
    free(iv->gidx);
}

/* Entries keyed by destination (directed graphs), in (node, slot) order,
 * with timestamp groups inside each node's segment. */
static int build_inview(const orc *o, orc_inview *iv)
{
    int64_t m = o->m, N = o->n_nodes;
    memset(iv, 0, sizeof(*iv));
    orc_entry *ent = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(m > 0 ? m : 1));
    iv->order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    iv->off = (int64_t *)calloc((size_t)(N + 1), sizeof(int64_t));
    iv->group_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    iv->gidx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (!ent || !iv->order || !iv->off || !iv->group_off || !iv->gidx) {
        free(ent);
        free_inview(iv);
        return ORC_ENOMEM;
    }
    for (int64_t p = 0; p < m; p++) {
        ent[p].node = o->live[p].dst;
        ent[p].slot = p;
    }
    qsort(ent, (size_t)m, sizeof(orc_entry), cmp_entry);
    for (int64_t i = 0; i < m; i++) {
        iv->order[i] = ent[i].slot;
        iv->off[ent[i].node + 1] += 1;
    }
    for (int64_t v = 0; v < N; v++) iv->off[v + 1] += iv->off[v];
    int64_t Gn = 0;
    for (int64_t v = 0; v < N; v++) {
        iv->gidx[v] = Gn;
        for (int64_t i = iv->off[v]; i < iv->off[v + 1]; i++)
            if (i == iv->off[v] || o->live[iv->order[i]].ts != o->live[iv->order[i - 1]].ts)
                iv->group_off[Gn++] = i;
    }
    iv->gidx[N] = Gn;
    iv->group_off[Gn] = m;
    iv->Gn = Gn;
    free(ent);
    return ORC_OK;
}

/* the far endpoint and timestamp of in-view entry slot */
static int64_t back_other(const orc *o, int64_t slot)
{
    return o->directed ? o->live[slot].src : slot_other(o, slot);
}

static int32_t one_walk_back(const orc *o, const orc_inview *iv, const orc_pairs *P, uint64_t w, int32_t max_len,
                             int bias, int start_policy, int64_t start_node, uint64_t seed, int32_t *node,
                             int64_t *tsout, double *margin, double lambda_start, double *bytes)
{
    for (int32_t i = 0; i < max_len; i++) {
        node[i] = -1;
        tsout[i] = INT64_MIN;
        if (margin) margin[i] = INFINITY;
    }
    if (o->m == 0) return 0;
    uint32_t r[4];
    double u1, u2;
    int32_t len;
    int64_t v, t;
    int64_t prev = -1;
    if (start_policy == START_PER_NODE) {
        node[0] = (int32_t)start_node;
        len = 1;
        v = start_node;
        t = INT64_MAX;
    } else {
        walk_block(seed, w, 0, r);
        u1 = orc_u53(r[0], r[1]);
        u2 = orc_u53(r[2], r[3]);
        int64_t k;
        if (start_policy == START_UNIFORM_EDGE) {
            k = o->m - 1 - uniform_index(u1, o->m);
        } else {
            const int sb = bias == BIAS_NODE2VEC ? BIAS_EXP : bias;
            int64_t g = o->G_tot - 1 - orc_sampler_index(u1, o->G_tot, sb, lambda_start);
            if (margin && sb != BIAS_UNIFORM) margin[1] = draw_margin(u1, o->G_tot, sb, lambda_start);
            int64_t a = o->ts_group_off[g], size = o->ts_group_off[g + 1] - a;
            k = a + size - 1 - uniform_index(u2, size);
        }
        int32_t a = o->live[k].dst, b = o->live[k].src;
        if (!o->directed && (r[3] & 1u)) {
            int32_t tmp = a; a = b; b = tmp;
        }
        node[0] = a;
        node[1] = b;
        tsout[1] = o->live[k].ts;
        len = 2;
        if (bytes) *bytes += 3 * 32.0 + 4 + 4 + 8 + 8 + 4;
        prev = a;
        v = b;
        t = o->live[k].ts;
    }
    while (len < max_len) {
        const uint32_t h = (uint32_t)(len - 1);
        const int64_t g0 = iv->gidx[v], g1 = iv->gidx[v + 1];
        /* c: first group at or after t; Gamma^- = groups [g0, c) */
        int64_t lo = g0, hi = g1;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (slot_ts(o, iv->order[iv->group_off[mid]]) >= t) hi = mid;
            else lo = mid + 1;
        }
        const int64_t c = lo;
        if (c == g0) break; /* Gamma^-_t(v) is empty */
        if (bias == BIAS_NODE2VEC) {
            const int64_t slot = n2v_pick(o, P, iv->group_off, iv->order, g0, c, 1, prev, seed, w, h,
                                          margin ? &margin[len] : NULL, bytes);
            if (slot < 0) break; /* every proposal rejected */
            node[len] = (int32_t)back_other(o, slot);
            tsout[len] = slot_ts(o, slot);
            if (bytes) {
                int64_t G = g1 - g0;
                int lg = 0;
                while (((int64_t)1 << lg) < G + 1) lg++;
                int search = lg - 2 > 1 ? lg - 2 : 1;
                *bytes += 32.0 * (1 + search + 1) + 12 + 16;
            }
            prev = v;
            v = node[len];
            t = tsout[len];
            len++;
            continue;
        }
        walk_block(seed, w, h, r);
        u1 = orc_u53(r[0], r[1]);
        u2 = orc_u53(r[2], r[3]);
        int64_t idx;
        if (bias == BIAS_UNIFORM) {
            int64_t e0 = iv->group_off[g0], e1 = iv->group_off[c];
            idx = e1 - 1 - uniform_index(u1, e1 - e0);
        } else {
            int64_t n = c - g0;
            int64_t j = orc_sampler_index(u1, n, bias, o->lambda_hop);
            if (margin) margin[len] = draw_margin(u1, n, bias, o->lambda_hop);
            int64_t gg = c - 1 - j;
            int64_t e0 = iv->group_off[gg], e1 = iv->group_off[gg + 1];
            idx = e1 - 1 - uniform_index(u2, e1 - e0);
        }
        int64_t slot = iv->order[idx];
        node[len] = (int32_t)back_other(o, slot);
        tsout[len] = slot_ts(o, slot);
        if (bytes) {
            int64_t G = g1 - g0;
            int lg = 0;
            while (((int64_t)1 << lg) < G + 1) lg++;
            int search = lg - 2 > 1 ? lg - 2 : 1;
            *bytes += 32.0 * (1 + search + 1) + 12 + 16;
        }
        prev = v;
        v = node[len];
        t = tsout[len];
        len++;
    }
    return len;
}

/* ------------------------------------------------------------------ */
/* Temporal Node2Vec (Sec. 2.5).                                      */
/* ------------------------------------------------------------------ */
/*
 * The second-order factor beta(u, w) of a candidate w, reached from the
 * current node whose predecessor on the walk is u (node2vec's return and
 * in-out parameters p, q): 1/p when w is u, 1 when w is a neighbour of u,
 * 1/q otherwise.  Reading: w is a neighbour of u when the window holds a live
 * edge u -> w (either orientation for undirected graphs); a backward walk
 * walks the time-reversed graph, whose edge u -> w is the live edge w -> u.
 * Each hop draws a proposal from the exponential sampler over the candidate
 * groups (then an edge uniformly inside the group) and accepts it with
 * probability beta / beta_max, beta_max = max(1/p, 1, 1/q); a rejected
 * proposal is drawn again.  Proposal k of the hop uses Philox word 1 = k
 * (proposal 0 is the plain exponential draw), its acceptance uniform the block
 * with word 1 = 2^31 + k; a proposal whose beta equals beta_max is accepted
 * without one.  After N2V_MAX_TRIALS rejections the walk ends.
 */
static int cmp_u64(const void *a, const void *b)
{
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int build_pairs(const orc *o, orc_pairs *P)
{
    const int64_t n = o->directed ? o->m : 2 * o->m;
    P->key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    P->n = 0;
    if (!P->key) return ORC_ENOMEM;
    for (int64_t p = 0; p < o->m; p++) {
        const uint64_t a = (uint64_t)(uint32_t)o->live[p].src, b = (uint64_t)(uint32_t)o->live[p].dst;
        P->key[P->n++] = a << 32 | b;
        if (!o->directed) P->key[P->n++] = b << 32 | a;
    }
    qsort(P->key, (size_t)P->n, sizeof(uint64_t), cmp_u64);
    return ORC_OK;
}

static int pair_live(const orc_pairs *P, int64_t from, int64_t to)
{
    const uint64_t k = (uint64_t)(uint32_t)from << 32 | (uint64_t)(uint32_t)to;
    int64_t lo = 0, hi = P->n;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (P->key[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo < P->n && P->key[lo] == k;
}

/*
 * One Node2Vec hop over the candidate groups [lo, hi) of a node view
 * (group_off, order): forward walks index them from lo, backward walks from
 * hi - 1 with mirrored edges inside a group.  prev < 0 (a PER_NODE start)
 * accepts the first proposal.  Returns the chosen slot, or -1 when every
 * proposal was rejected.  margin (nullable) receives the smallest sampler
 * margin over the proposals drawn; bytes adds 12 + 16 per proposal after the
 * first and 32 per adjacency lookup (the sector model of the extra reads).
 */
static int64_t n2v_pick(const orc *o, const orc_pairs *P, const int64_t *group_off, const int64_t *order, int64_t lo,
                        int64_t hi, int back, int64_t prev, uint64_t seed, uint64_t w, uint32_t h, double *margin,
                        double *bytes)
{
    const double inv_p = 1.0 / o->n2v_p, inv_q = 1.0 / o->n2v_q;
    double bmax = inv_p > 1.0 ? inv_p : 1.0;
    if (inv_q > bmax) bmax = inv_q;
    const int64_t n = hi - lo;
    double mg = INFINITY;
    for (uint32_t k = 0; k < N2V_MAX_TRIALS; k++) {
        uint32_t r[4];
        draw_block(seed, w, h, k, r);
        const double u1 = orc_u53(r[0], r[1]), u2 = orc_u53(r[2], r[3]);
        const int64_t j = orc_sampler_index(u1, n, BIAS_EXP, o->lambda_hop);
        const double m1 = draw_margin(u1, n, BIAS_EXP, o->lambda_hop);
        if (m1 < mg) mg = m1;
        if (k > 0 && bytes) *bytes += 12 + 16;
        const int64_t gg = back ? hi - 1 - j : lo + j;
        const int64_t e0 = group_off[gg], e1 = group_off[gg + 1];
        const int64_t q = uniform_index(u2, e1 - e0);
        const int64_t slot = order[back ? e1 - 1 - q : e0 + q];
        if (prev < 0) {
            if (margin) *margin = mg;
            return slot;
        }
        const int64_t cand = back ? back_other(o, slot) : slot_other(o, slot);
        double beta;
        if (cand == prev) {
            beta = inv_p;
        } else if (inv_q == 1.0) {
            beta = 1.0; /* a neighbour or not, the factor is 1 */
        } else {
            if (bytes) *bytes += 32;
            const int adj = back ? pair_live(P, cand, prev) : pair_live(P, prev, cand);
            beta = adj ? 1.0 : inv_q;
        }
        int accept = beta >= bmax;
        if (!accept) {
            draw_block(seed, w, h, 0x80000000u | k, r);
            accept = orc_u53(r[0], r[1]) * bmax < beta;
        }
        if (accept) {
            if (margin) *margin = mg;
            return slot;
        }
    }
    if (margin) *margin = mg;
    return -1;
}

static double eff_lambda_start(const orc *o)
{
    if (o->lambda_start > 0.0) return o->lambda_start;
    return o->G_tot > 0 ? 1.0 / (double)o->G_tot : 1.0;
}

/*
 * Walks for walk ids ids[0..n) (or 0..n when ids is NULL).  bias / max_len
 * per walk come from the arrays when given, else from the scalars.  Outputs
 * are row-major [n][max_len_cap].
 */
int orc_walks(const orc *o, int64_t n, const int64_t *ids, int32_t max_len_cap,
              const int32_t *max_len_arr, int32_t max_len, const uint8_t *bias_arr, int bias,
              int start_policy, int64_t walks_per_node, int direction, uint64_t seed, int32_t *node, int64_t *ts,
              int32_t *len, double *margin, double *bytes)
{
    if (n < 0 || max_len_cap < 2 || direction < 0 || direction > 1) return ORC_EINVAL;
    /* backward walks: the in-view (the out-view itself for undirected graphs) */
    orc_inview iv;
    int have_iv = 0;
    if (direction == 1) {
        if (o->directed) {
            int rc = build_inview(o, &iv);
            if (rc) return rc;
            have_iv = 1;
        } else {
            iv.off = o->node_off;
            iv.order = o->node_order;
            iv.group_off = o->node_group_off;
            iv.gidx = o->node_gidx;
            iv.Gn = o->Gn;
        }
    }
#define ORC_WALKS_FAIL(code) do { if (have_iv) free_inview(&iv); return (code); } while (0)
    if (start_policy != START_UNIFORM_EDGE && start_policy != START_BIASED_TS && start_policy != START_PER_NODE)
        ORC_WALKS_FAIL(ORC_EINVAL);
    int32_t *active = NULL;
    int64_t n_active = 0;
    if (start_policy == START_PER_NODE && o->m > 0) {
        if (walks_per_node < 1) ORC_WALKS_FAIL(ORC_EINVAL);
        const int64_t *gx = direction == 1 ? iv.gidx : o->node_gidx;
        for (int64_t v = 0; v < o->n_nodes; v++) n_active += gx[v + 1] > gx[v];
        active = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_active > 0 ? n_active : 1));
        if (!active) ORC_WALKS_FAIL(ORC_ENOMEM);
        n_active = 0;
        for (int64_t v = 0; v < o->n_nodes; v++)
            if (gx[v + 1] > gx[v]) active[n_active++] = (int32_t)v;
    }
    /* live pairs for Node2Vec adjacency tests, when a walk takes that bias */
    orc_pairs pairs = {NULL, 0};
    int want_pairs = bias_arr == NULL && bias == BIAS_NODE2VEC;
    for (int64_t i = 0; bias_arr && i < n && !want_pairs; i++) want_pairs = bias_arr[i] == BIAS_NODE2VEC;
    if (want_pairs && build_pairs(o, &pairs)) {
        free(active);
        ORC_WALKS_FAIL(ORC_ENOMEM);
    }
    double ls = eff_lambda_start(o);
    if (bytes) *bytes = 0.0;
    for (int64_t i = 0; i < n; i++) {
        uint64_t w = ids ? (uint64_t)ids[i] : (uint64_t)i;
        int32_t L = max_len_arr ? max_len_arr[i] : max_len;
        int b = bias_arr ? (int)bias_arr[i] : bias;
        if (L < 2 || L > max_len_cap || b < 0 || b > 4 || (direction == 1 && b == BIAS_EXP_WEIGHT)) {
            free(active);
            free(pairs.key);
            ORC_WALKS_FAIL(ORC_EINVAL);
        }
        int64_t start_node = -1;
        if (active) {
            const int64_t a = (int64_t)(w / (uint64_t)walks_per_node);
            if (a >= n_active) {
                free(active);
                free(pairs.key);
                ORC_WALKS_FAIL(ORC_EINVAL);
            }
            start_node = active[a];
        }
        int32_t *nr = node + i * (int64_t)max_len_cap;
        int64_t *tr = ts + i * (int64_t)max_len_cap;
        double *mr = margin ? margin + i * (int64_t)max_len_cap : NULL;
        for (int32_t j = L; j < max_len_cap; j++) {
            nr[j] = -1;
            tr[j] = INT64_MIN;
            if (mr) mr[j] = INFINITY;
        }
        if (direction == 1)
            len[i] = one_walk_back(o, &iv, &pairs, w, L, b, start_policy, start_node, seed, nr, tr, mr, ls, bytes);
        else
            len[i] = one_walk(o, &pairs, w, L, b, start_policy, start_node, seed, nr, tr, mr, ls, bytes);
    }
    free(active);
    free(pairs.key);
    if (have_iv) free_inview(&iv);
#undef ORC_WALKS_FAIL
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* State export (canonical form compared against the CUDA library).   */
/* ------------------------------------------------------------------ */
void orc_counts(const orc *o, int64_t out[10])
{
    out[0] = o->m;
    out[1] = o->G_tot;
    out[2] = o->n_nodes;
    out[3] = o->M;
    out[4] = o->Gn;
    out[5] = o->dropped_late;
    out[6] = o->evicted;
    out[7] = o->has_cutoff;
    out[8] = o->cutoff;
    out[9] = o->seq_next;
}

/* live edges: src, dst, ts in store order (m each) */
void orc_export_live(const orc *o, int32_t *src, int32_t *dst, int64_t *ts)
{
    for (int64_t i = 0; i < o->m; i++) {
        src[i] = o->live[i].src;
        dst[i] = o->live[i].dst;
        ts[i] = o->live[i].ts;
    }
}

void orc_export_ts_groups(const orc *o, int64_t *off /* G_tot + 1 */)
{
    memcpy(off, o->ts_group_off, sizeof(int64_t) * (size_t)(o->G_tot + 1));
}

void orc_export_node_view(const orc *o, int64_t *node_off /* N+1 */, int64_t *node_order /* M */,
                          int64_t *node_group_off /* Gn+1 */, int64_t *node_gidx /* N+1 */)
{
    memcpy(node_off, o->node_off, sizeof(int64_t) * (size_t)(o->n_nodes + 1));
    if (o->M) memcpy(node_order, o->node_order, sizeof(int64_t) * (size_t)o->M);
    memcpy(node_group_off, o->node_group_off, sizeof(int64_t) * (size_t)(o->Gn + 1));
    memcpy(node_gidx, o->node_gidx, sizeof(int64_t) * (size_t)(o->n_nodes + 1));
}
