"""Pins of the CPU oracle against things other than itself.

* Philox4x32-10 against cuRAND's host-side generator (an independent library
  implementation of the same published generator), for the exact counters the
  walks use.
* The samplers against the inverse-CDF property of the weights of Sec. 2.5
  (exact rationals / 80-digit decimals), against the hand-worked example, and
  by chi-square on their output frequencies.
* The index state against a hand-worked fixture and against brute force from
  the window-set and view definitions (Sec. 2.3, 2.6) on random tiny streams.
* Whole walks against exact enumeration of walk probabilities on tiny graphs
  (chi-square), and against the causality invariants.
"""
import ctypes
import ctypes.util
import glob
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import brute
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def _find_curand():
    cands = []
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        cands += sorted(glob.glob(os.path.join(d, "libcurand.so*")))
    try:
        import nvidia  # noqa: F401
        for p in nvidia.__path__:
            cands += sorted(glob.glob(os.path.join(p, "**", "libcurand.so*"), recursive=True))
    except Exception:
        pass
    f = ctypes.util.find_library("curand")
    if f:
        cands.append(f)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_block(L, seed, block):
    """Block `block` of cuRAND's host Philox4x32-10 stream for `seed`."""
    gen = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_uint64(seed)) == 0
        assert L.curandSetGeneratorOffset(gen, ctypes.c_uint64(4 * block)) == 0
        out = (ctypes.c_uint32 * 4)()
        assert L.curandGenerate(gen, out, ctypes.c_size_t(4)) == 0
        return [int(x) for x in out]
    finally:
        L.curandDestroyGenerator(gen)


def test_philox_matches_curand_host_generator():
    L = _find_curand()
    if L is None:
        pytest.skip("libcurand not found")
    # cuRAND's host stream visits counter (B >> 16, 0, B & 0xffff, 0) at block
    # B; the walks use counter (hop, 0, walk, 0) -> block hop * 65536 + walk.
    rng = random.Random(7)
    cases = [(0, 0, 0), (0, 1, 0), (0x123456789abcdef, 0, 0), (2**64 - 1, 79, 65535)]
    cases += [(rng.getrandbits(64), rng.randrange(0, 100), rng.randrange(0, 65536)) for _ in range(40)]
    for seed, hop, walk in cases:
        want = _curand_host_block(L, seed, hop * 65536 + walk)
        got = O.philox4x32_10([hop, 0, walk, 0], [seed & 0xffffffff, seed >> 32])
        assert [int(x) for x in got] == want, (seed, hop, walk)


def test_u53_range():
    assert O.u53(0, 0) == 0.0
    assert O.u53(0xffffffff, 0xffffffff) == 1.0 - 2.0 ** -53
    assert O.u53(0x80000000, 0) == 0.5
    # the low 11 bits of the second word do not enter u
    assert O.u53(0x12345678, 0x9abcdef0) == O.u53(0x12345678, 0x9abcdef0 | 0x7ff)


# ---------------------------------------------------------------- samplers
def _check_cdf_property(i, u, n, bias, lam):
    """CDF(i-1) <= u < CDF(i) for the exact distribution."""
    uf = Fraction(u)
    if bias in (0, 1):
        lo = brute.cdf_exact(i - 1, n, bias) if i > 0 else Fraction(0)
        hi = brute.cdf_exact(i, n, bias)
        return lo <= uf < hi, min(abs(uf - lo), abs(hi - uf))
    from decimal import Decimal
    ud = Decimal(uf.numerator) / Decimal(uf.denominator)
    lo = brute.cdf_exact(i - 1, n, bias, lam) if i > 0 else Decimal(0)
    hi = brute.cdf_exact(i, n, bias, lam)
    return lo <= ud < hi, min(abs(ud - lo), abs(hi - ud))


@pytest.mark.parametrize("bias", [0, 1, 2])
def test_sampler_inverse_cdf_property(bias):
    rng = random.Random(100 + bias)
    bad = 0
    for trial in range(3000):
        n = rng.choice([1, 2, 3, 5, 17, 100, 1000, rng.randrange(1, 5000)])
        lam = rng.choice([1.0, 0.5, 0.01, 1.0 / max(n, 1), 3.0]) if bias == 2 else 1.0
        u = rng.random()
        i = O.sampler_index(u, n, bias, lam)
        assert 0 <= i < n
        ok, dist = _check_cdf_property(i, u, n, bias, lam)
        if not ok:
            # only allowed within rounding distance of a bucket boundary
            assert float(dist) < 1e-12, (bias, n, lam, u, i)
            bad += 1
    assert bad <= 3


def test_sampler_extreme_u():
    for bias in (0, 1, 2):
        for n in (1, 2, 7, 10**6, 2**31 - 1):
            assert O.sampler_index(0.0, n, bias, 1.0) == 0
            assert O.sampler_index(1.0 - 2.0 ** -53, n, bias, 1.0) == n - 1
    # n == 1 always draws index 0
    for u in (0.0, 0.3, 0.999):
        for bias in (0, 1, 2):
            assert O.sampler_index(u, 1, bias, 1.0) == 0


def test_printed_eq3_is_off_by_one_but_oracle_is_not():
    """The printed exponential sampler floor(n + ln u - 1) never returns n-1,
    which the inverse-CDF pin rejects; the oracle's exact form passes."""
    n, u = 10, 0.9
    printed = math.floor(n + math.log(u) - 1)
    ok, _ = _check_cdf_property(printed, u, n, 2, 1.0)
    assert not ok
    i = O.sampler_index(u, n, 2, 1.0)
    assert i == n - 1
    assert _check_cdf_property(i, u, n, 2, 1.0)[0]


def test_sampler_worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "tiny_stream.json")))["sampler_example"]
    for bias_name, bias in (("linear", 1), ("exp", 2)):
        for u, want in ex["group_index_at_u"][bias_name]:
            assert O.sampler_index(u, 2, bias, 1.0) == want, (bias_name, u)
    # x lands exactly on the boundary for linear at u = 1/3
    assert O.sampler_x(1.0 / 3.0, 2, 1, 1.0) == 1.0


@pytest.mark.parametrize("bias,n,lam", [(0, 7, 1.0), (1, 6, 1.0), (2, 5, 1.0), (2, 40, 0.1)])
def test_sampler_chi_square(bias, n, lam):
    from scipy.stats import chisquare
    draws = 200_000
    counts = np.zeros(n, np.int64)
    for k in range(draws):
        r = O.philox4x32_10([k & 0xffffffff, 0, 5, 0], [123, 456])
        counts[O.sampler_index(O.u53(r[0], r[1]), n, bias, lam)] += 1
    w = np.array(brute.group_weights(n, bias, lam), np.float64)
    exp = w / w.sum() * draws
    keep = exp > 5
    stat, p = chisquare(counts[keep], exp[keep] * counts[keep].sum() / exp[keep].sum())
    assert p > 1e-3, (p, counts, exp)


# ---------------------------------------------------------------- index state
def _state_equal(st, want, directed=True):
    for k in ("src", "dst", "ts", "ts_group_off", "node_off", "node_order", "node_group_off",
              "node_gidx"):
        assert list(st[k]) == list(want[k]), k
    assert st["counts"]["dropped_late"] == want["dropped_late"]
    assert st["counts"]["evicted"] == want["evicted"]
    if want.get("cutoff") is not None:
        assert st["counts"]["has_cutoff"] == 1
        assert st["counts"]["cutoff"] == want["cutoff"]


def test_state_hand_worked_fixture():
    fx = json.load(open(os.path.join(GOLDEN, "tiny_stream.json")))
    o = O.Oracle(window=fx["window"], directed=fx["directed"])
    for b, want in zip(fx["batches"], fx["expected"]):
        o.ingest(b["src"], b["dst"], b["ts"])
        _state_equal(o.state(), want)


def _random_stream(rng, n_batches, max_batch, n_nodes, ts_span, monotone):
    out = []
    t = 0
    for _ in range(n_batches):
        k = rng.randrange(0, max_batch + 1)
        src = [rng.randrange(0, n_nodes) for _ in range(k)]
        dst = [rng.randrange(0, n_nodes) for _ in range(k)]
        if monotone:
            ts = []
            for _ in range(k):
                t += rng.choice([0, 0, 1, 2, 5])
                ts.append(t)
        else:
            ts = [rng.randrange(-ts_span // 4, ts_span) + t for _ in range(k)]
            t += ts_span // 3
        out.append((src, dst, ts))
    return out


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("window", [0, 6, 25, -1, -7, -30])
def test_state_matches_brute_force(directed, window):
    rng = random.Random(hash((directed, window)) & 0xffff)
    for trial in range(25):
        stream = _random_stream(rng, rng.randrange(1, 6), 12, rng.randrange(1, 7), 20,
                                monotone=rng.random() < 0.4)
        want = brute.window_state(stream, window, directed)
        o = O.Oracle(window=window, directed=directed)
        for (s, d, t), w in zip(stream, want):
            o.ingest(s, d, t)
            st = o.state()
            _state_equal(st, w, directed)
            assert st["counts"]["n_nodes"] == w["n_nodes"]


def test_ingest_rejects_bad_input():
    o = O.Oracle(window=0)
    with pytest.raises(ValueError):
        o.ingest([0, -1], [1, 1], [1, 2])
    assert o.counts()["m"] == 0
    o.ingest([], [], [])
    assert o.counts()["m"] == 0


def test_undirected_view_is_symmetric():
    """Swapping src and dst of every edge leaves the undirected node view's
    (node, other, ts) multiset unchanged."""
    rng = random.Random(3)
    s = [rng.randrange(0, 6) for _ in range(40)]
    d = [rng.randrange(0, 6) for _ in range(40)]
    t = [rng.randrange(0, 10) for _ in range(40)]

    def view(a, b):
        o = O.Oracle(window=0, directed=False)
        o.ingest(a, b, t)
        st = o.state()
        res = []
        for v in range(len(st["node_off"]) - 1):
            for i in range(st["node_off"][v], st["node_off"][v + 1]):
                slot = st["node_order"][i]
                p = slot >> 1
                other = st["src"][p] if slot & 1 else st["dst"][p]
                res.append((v, int(other), int(st["ts"][p])))
        return sorted(res)

    assert view(s, d) == view(d, s)


# ---------------------------------------------------------------- walks
def _walk_key(node_row, ts_row, ln):
    return tuple((int(node_row[i]), None if i == 0 else int(ts_row[i])) for i in range(ln))


@pytest.mark.parametrize("directed,bias,policy", [
    (True, 0, 0), (True, 1, 0), (True, 2, 0), (True, 1, 1), (True, 2, 1), (True, 0, 1),
    (False, 0, 0), (False, 2, 1), (True, 3, 0), (False, 3, 1),
])
def test_walk_distribution_matches_enumeration(directed, bias, policy):
    from scipy.stats import chisquare
    # tiny graph with ties, a self-loop and a dead end
    src = [0, 0, 0, 1, 1, 2, 2, 3, 0, 2]
    dst = [1, 2, 1, 2, 0, 0, 3, 0, 0, 2]
    ts = [1, 2, 2, 3, 4, 5, 5, 6, 7, 6]
    lam_hop, lam_start = 0.7, 0.4
    max_len = 4
    lam_w = 0.45
    o = O.Oracle(window=0, directed=directed)
    o.ingest(src, dst, ts)
    o.set_bias_params(lam_hop, lam_start)
    o.set_weight_rate(lam_w)
    live = brute.window_state([(src, dst, ts)], 0, directed)[-1]["live"]
    dist = brute.walk_distribution(live, directed, max_len, bias, policy, lam_hop, lam_start, lam_w=lam_w)
    assert abs(sum(dist.values()) - 1.0) < 1e-9
    n = 60_000
    node, tsa, ln, _, _ = o.walks(n, max_len, bias=bias, start_policy=policy, seed=99)
    counts = {}
    for i in range(n):
        k = _walk_key(node[i], tsa[i], ln[i])
        assert k in dist, k
        counts[k] = counts.get(k, 0) + 1
    keys = [k for k in dist if dist[k] * n > 5]
    obs = np.array([counts.get(k, 0) for k in keys], np.float64)
    exp = np.array([dist[k] * n for k in keys], np.float64)
    exp *= obs.sum() / exp.sum()
    stat, p = chisquare(obs, exp)
    assert p > 1e-3, p


@pytest.mark.parametrize("directed,bias", [(True, 0), (True, 1), (True, 2), (False, 2)])
def test_per_node_walks_match_enumeration(directed, bias):
    """K walks start at every node with a live edge, in id order; each start
    node's walks follow the exact walk distribution from that node, whose
    first hop may take any live edge of the node."""
    from scipy.stats import chisquare
    src = [0, 0, 0, 1, 1, 2, 2, 3, 0, 2, 5]
    dst = [1, 2, 1, 2, 0, 0, 3, 0, 0, 2, 1]
    ts = [1, 2, 2, 3, 4, 5, 5, 6, 7, 6, 3]
    lam_hop = 0.7
    max_len = 4
    o = O.Oracle(window=0, directed=directed)
    o.ingest(src, dst, ts)
    o.set_bias_params(lam_hop, 0.4)
    act = list(o.active_nodes())
    want = sorted(set(src) | (set() if directed else set(dst)))
    assert act == want  # node 4 has no edge; 5 only an out-edge
    live = brute.window_state([(src, dst, ts)], 0, directed)[-1]["live"]
    K = 12_000
    node, tsa, ln, _, _ = o.walks(K * len(act), max_len, bias=bias, start_policy=O.START_PER_NODE, seed=5)
    assert (ln >= 2).all()  # an active node always has a first hop
    for a, v in enumerate(act):
        dist = brute.walk_distribution(live, directed, max_len, bias, 0, lam_hop, 0.4, start_node=v)
        assert abs(sum(dist.values()) - 1.0) < 1e-9
        counts = {}
        for i in range(a * K, (a + 1) * K):
            assert node[i][0] == v and tsa[i][0] == np.iinfo(np.int64).min
            k = _walk_key(node[i], tsa[i], ln[i])
            assert k in dist, k
            counts[k] = counts.get(k, 0) + 1
        keys = [k for k in dist if dist[k] * K > 5]
        if len(keys) < 2:
            continue
        obs = np.array([counts.get(k, 0) for k in keys], np.float64)
        exp = np.array([dist[k] * K for k in keys], np.float64)
        exp *= obs.sum() / exp.sum()
        assert chisquare(obs, exp)[1] > 1e-3, v


# ------------------------------------------------- weight-based sampler (Sec. 2.5)
@pytest.mark.parametrize("lam", [1.0, 0.3, 2.5])
def test_weight_sampler_worked_example(lam):
    """Node with live edges at ts {1, 2, 2, 5}, t = 1: Gamma holds the two
    edges at 2 and the one at 5; weights exp(lam (ts - 2)) give group 0 the
    probability 2 / (2 + e^{3 lam}), so u below that picks group 0."""
    b = 2.0 / (2.0 + math.exp(3.0 * lam))
    for u, want in ((0.0, 0), (b * (1 - 1e-9), 0), (b * (1 + 1e-9), 1), (0.999999, 1), (b / 2, 0)):
        j, mg = O.weight_pick([2, 5], [2, 1], lam, u)
        assert j == want, (u, j)
    # the margin measures the distance to the boundary
    assert O.weight_pick([2, 5], [2, 1], lam, b * (1 + 1e-9))[1] < 1e-8


def test_weight_sampler_frequencies_and_invariances():
    from scipy.stats import chisquare
    rng = np.random.default_rng(4)
    for trial in range(6):
        n = int(rng.integers(2, 12))
        ts = np.cumsum(rng.integers(1, 50, n)).astype(np.int64)
        size = rng.integers(1, 4, n).astype(np.int64)
        lam = float(rng.choice([0.001, 0.02, 0.1]))
        w = size * np.exp(lam * (ts - ts[0]).astype(np.float64))
        p = w / w.sum()
        us = rng.random(20000)
        picks = np.array([O.weight_pick(ts, size, lam, u)[0] for u in us])
        obs = np.bincount(picks, minlength=n).astype(np.float64)
        keep = p * len(us) > 5
        exp = p * len(us)
        assert chisquare(obs[keep], exp[keep] * obs[keep].sum() / exp[keep].sum())[1] > 1e-3
        # shifting every timestamp changes nothing; the pick is the inverse CDF
        for u in us[:200]:
            j = O.weight_pick(ts, size, lam, u)[0]
            assert O.weight_pick(ts + 10**12, size, lam, u)[0] == j
            cdf = np.cumsum(p)
            assert j == int(np.searchsorted(cdf, u * (1 - 1e-12), "left")) or abs(cdf[j - 1] - u) < 1e-9
    # a rate whose raw weights overflow exp (lambda (t_max - t_min) = 3000)
    # still gives the limit: all mass on the newest group, a finite margin
    j, mg = O.weight_pick([0, 10, 30000], [5, 5, 1], 0.1, 0.999)
    assert j == 2 and math.isfinite(mg)
    # a vanishing rate weighs every edge the same
    j = [O.weight_pick([0, 7, 9], [1, 2, 1], 1e-15, u)[0] for u in (0.2, 0.3, 0.7, 0.8)]
    assert j == [0, 1, 1, 2]


def test_per_node_walks_need_a_whole_number_per_node():
    o = O.Oracle(window=0, directed=True)
    o.ingest([0, 1, 2], [1, 2, 0], [1, 2, 3])
    with pytest.raises(ValueError):
        o.walks(7, 4, start_policy=O.START_PER_NODE)  # 3 active nodes
    node, _, ln, _, _ = o.walks(6, 4, start_policy=O.START_PER_NODE)
    assert list(node[:, 0]) == [0, 0, 1, 1, 2, 2]


def test_int64_min_timestamps_are_rejected():
    o = O.Oracle(window=0, directed=True)
    with pytest.raises(Exception):
        o.ingest([0], [1], [np.iinfo(np.int64).min])


def _check_walk_invariants(st, directed, node, tsa, ln, max_len):
    live = {}
    for a, b, t in zip(st["src"], st["dst"], st["ts"]):
        live[(int(a), int(b), int(t))] = live.get((int(a), int(b), int(t)), 0) + 1
        if not directed:
            live[(int(b), int(a), int(t))] = live.get((int(b), int(a), int(t)), 0) + 1
    # per node: sorted ts of its entries, for the termination check
    by_node = {}
    for (a, b, t) in live:
        by_node.setdefault(a, []).append(t)
    for v in by_node:
        by_node[v].sort()
    for i in range(node.shape[0]):
        L = int(ln[i])
        assert 2 <= L <= max_len
        for h in range(1, L):
            e = (int(node[i, h - 1]), int(node[i, h]), int(tsa[i, h]))
            assert e in live, (i, h, e)
            if h >= 2:
                assert tsa[i, h] > tsa[i, h - 1]
        assert (node[i, L:] == -1).all() and (tsa[i, L:] == np.iinfo(np.int64).min).all()
        if L < max_len:  # stopped early: no continuation exists
            v, t = int(node[i, L - 1]), int(tsa[i, L - 1])
            assert not any(x > t for x in by_node.get(v, [])), (i, v, t)


@pytest.mark.parametrize("directed", [True, False])
def test_walk_invariants_small_config(directed):
    from paper_2605_16182_gb300 import synth
    spec = synth.config_small(scale=0.05)
    o = O.Oracle(window=0, directed=directed)
    for k, s, d, t in spec.batches():
        o.ingest(s.numpy(), d.numpy(), t.numpy())
    st = o.state()
    for bias in (0, 1, 2):
        node, tsa, ln, _, _ = o.walks(2000, 12, bias=bias, seed=bias)
        _check_walk_invariants(st, directed, node, tsa, ln, 12)


def test_walks_by_id_subset_equal_full_run():
    from paper_2605_16182_gb300 import synth
    spec = synth.config_small(scale=0.05)
    o = O.Oracle(window=0)
    for k, s, d, t in spec.batches():
        o.ingest(s.numpy(), d.numpy(), t.numpy())
    full = o.walks(500, 10, bias=2, seed=5)
    ids = np.array([3, 499, 0, 77, 77], np.int64)
    sub = o.walks(ids=ids, max_len=10, bias=2, seed=5)
    assert (sub[0] == full[0][ids]).all() and (sub[1] == full[1][ids]).all()
    assert (sub[2] == full[2][ids]).all()


def test_walks_on_empty_graph():
    o = O.Oracle(window=0)
    node, tsa, ln, _, _ = o.walks(4, 5, seed=1)
    assert (ln == 0).all() and (node == -1).all()


# ---------------------------------------------------------------- backward walks
def _reversed(src, dst, ts):
    """The time-reversed graph: every edge (u, v, t) as (v, u, -t), arriving
    in mirrored order (one batch)."""
    return list(dst[::-1]), list(src[::-1]), [-x for x in ts[::-1]]


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("policy", [0, 1, 2])
def test_backward_walks_are_forward_walks_of_the_reversed_graph(directed, policy):
    """Backward walks on G equal forward walks on the time-reversed graph,
    position by position, for every bias and start policy: the two run
    through different code (in-view search for the last earlier group vs the
    forward search) over mirrored data."""
    rng = np.random.default_rng(12 + directed)
    n = 400
    src = list(rng.integers(0, 25, n))
    dst = list(rng.integers(0, 25, n))
    ts = list(rng.integers(1, 60, n))  # many ties
    a = O.Oracle(window=0, directed=directed)
    a.ingest(src, dst, ts)
    b = O.Oracle(window=0, directed=directed)
    b.ingest(*_reversed(src, dst, ts))
    na = len(a.active_nodes(1))
    assert na == len(b.active_nodes())
    a.set_node2vec(0.5, 3.0)  # Node2Vec's neighbour test reverses with the graph
    b.set_node2vec(0.5, 3.0)
    for bias in (0, 1, 2, 4):
        nw = 5 * na if policy == 2 else 3000
        g = a.walks(nw, 9, bias=bias, start_policy=policy, seed=bias + 7, direction=1)
        f = b.walks(nw, 9, bias=bias, start_policy=policy, seed=bias + 7)
        assert np.array_equal(g[2], f[2]), (bias, policy)
        assert np.array_equal(g[0], f[0])
        imin = np.iinfo(np.int64).min
        real = g[1] != imin
        assert np.array_equal(g[1] != imin, f[1] != imin)
        assert np.array_equal(g[1][real], -f[1][real])


def test_backward_walks_follow_in_edges_back_in_time():
    rng = np.random.default_rng(3)
    src = list(rng.integers(0, 15, 300))
    dst = list(rng.integers(0, 15, 300))
    ts = list(rng.integers(1, 40, 300))
    o = O.Oracle(window=0, directed=True)
    o.ingest(src, dst, ts)
    edges = set(zip(src, dst, ts))
    node, tsa, ln, _, _ = o.walks(2000, 10, bias=2, seed=4, direction=1)
    for i in range(2000):
        for p in range(1, ln[i]):
            # position p was reached over the edge (node[p], node[p-1], ts[p])
            assert (int(node[i][p]), int(node[i][p - 1]), int(tsa[i][p])) in edges
            if p >= 2:
                assert tsa[i][p] < tsa[i][p - 1]
    with pytest.raises(ValueError):
        o.walks(10, 5, bias=3, direction=1)  # the weight-based bias runs forward only


# ------------------------------------------------------ Temporal Node2Vec (Sec. 2.5)
@pytest.mark.parametrize("directed,policy,pq", [
    (True, 0, (0.5, 2.0)), (True, 1, (4.0, 0.25)), (False, 0, (0.5, 2.0)), (False, 1, (2.0, 0.5)),
])
def test_node2vec_walks_match_enumeration(directed, policy, pq):
    """Rejection sampling on the exponential proposal gives the second-order
    law: each hop's exponential proposal reweighted by beta(prev, w) (1/p on
    a return, 1 to a neighbour of prev, 1/q otherwise) and normalised."""
    from scipy.stats import chisquare
    if directed:
        src = [0, 0, 0, 1, 1, 2, 2, 3, 0, 2, 3, 1]
        dst = [1, 2, 1, 2, 0, 0, 3, 0, 0, 2, 1, 3]
        ts = [1, 2, 2, 3, 4, 5, 5, 6, 7, 6, 7, 8]
    else:  # sparser, so that many candidates are not neighbours of the previous node
        src = [0, 1, 2, 1, 3, 4, 2, 5, 1, 3, 0, 4]
        dst = [1, 2, 3, 4, 0, 5, 5, 0, 2, 4, 1, 2]
        ts = [1, 2, 3, 3, 4, 4, 5, 6, 6, 7, 7, 8]
    lam_hop, lam_start, max_len = 0.7, 0.4, 4
    o = O.Oracle(window=0, directed=directed)
    o.ingest(src, dst, ts)
    o.set_bias_params(lam_hop, lam_start)
    o.set_node2vec(*pq)
    live = brute.window_state([(src, dst, ts)], 0, directed)[-1]["live"]
    dist = brute.walk_distribution(live, directed, max_len, 4, policy, lam_hop, lam_start, n2v=pq)
    assert abs(sum(dist.values()) - 1.0) < 1e-9
    # the second-order law differs from the first-order one on this graph
    first = brute.walk_distribution(live, directed, max_len, 2, policy, lam_hop, lam_start)
    assert sum(abs(dist.get(k, 0.0) - first.get(k, 0.0)) for k in set(dist) | set(first)) / 2 > 0.01
    n = 60_000
    node, tsa, ln, _, _ = o.walks(n, max_len, bias=4, start_policy=policy, seed=123)
    counts = {}
    for i in range(n):
        k = _walk_key(node[i], tsa[i], ln[i])
        assert k in dist, k
        counts[k] = counts.get(k, 0) + 1
    keys = [k for k in dist if dist[k] * n > 5]
    obs = np.array([counts.get(k, 0) for k in keys], np.float64)
    exp = np.array([dist[k] * n for k in keys], np.float64)
    exp *= obs.sum() / exp.sum()
    assert chisquare(obs, exp)[1] > 1e-3


@pytest.mark.parametrize("directed", [True, False])
def test_node2vec_per_node_first_hop_is_first_order(directed):
    """A PER_NODE walk has no predecessor at its first hop: that hop follows
    the exponential proposal; later hops the second-order law."""
    from scipy.stats import chisquare
    src = [0, 0, 0, 1, 1, 2, 2, 3, 0, 2, 5]
    dst = [1, 2, 1, 2, 0, 0, 3, 0, 0, 2, 1]
    ts = [1, 2, 2, 3, 4, 5, 5, 6, 7, 6, 3]
    pq = (0.4, 3.0)
    o = O.Oracle(window=0, directed=directed)
    o.ingest(src, dst, ts)
    o.set_bias_params(0.7, 0.4)
    o.set_node2vec(*pq)
    act = list(o.active_nodes())
    live = brute.window_state([(src, dst, ts)], 0, directed)[-1]["live"]
    K = 12_000
    node, tsa, ln, _, _ = o.walks(K * len(act), 4, bias=4, start_policy=O.START_PER_NODE, seed=6)
    for a, v in enumerate(act):
        dist = brute.walk_distribution(live, directed, 4, 4, 0, 0.7, 0.4, start_node=v, n2v=pq)
        counts = {}
        for i in range(a * K, (a + 1) * K):
            k = _walk_key(node[i], tsa[i], ln[i])
            assert k in dist, k
            counts[k] = counts.get(k, 0) + 1
        keys = [k for k in dist if dist[k] * K > 5]
        if len(keys) < 2:
            continue
        obs = np.array([counts.get(k, 0) for k in keys], np.float64)
        exp = np.array([dist[k] * K for k in keys], np.float64)
        exp *= obs.sum() / exp.sum()
        assert chisquare(obs, exp)[1] > 1e-3, v


@pytest.mark.parametrize("direction", [0, 1])
def test_node2vec_with_unit_parameters_is_the_exponential_walk(direction):
    """p = q = 1 makes every beta equal beta_max: every first proposal is
    accepted, and it is the exponential walk's own draw (Philox word 1 = 0)."""
    rng = np.random.default_rng(31)
    src, dst, ts = (list(rng.integers(0, 30, 500)), list(rng.integers(0, 30, 500)),
                    list(rng.integers(1, 80, 500)))
    for directed in (True, False):
        o = O.Oracle(window=0, directed=directed)
        o.ingest(src, dst, ts)
        o.set_node2vec(1.0, 1.0)
        for policy in (0, 1):
            a = o.walks(2000, 10, bias=4, start_policy=policy, seed=3, direction=direction)
            b = o.walks(2000, 10, bias=2, start_policy=policy, seed=3, direction=direction)
            for x, y in zip(a[:3], b[:3]):
                assert np.array_equal(x, y)


def test_node2vec_rejection_cap():
    """Edges 0 -> 1 (t 1) and 1 -> 0 (t 2): from 1, reached over 0 -> 1, the
    only candidate returns to 0, accepted with probability (1/p) / 1 = 1e-3;
    after 4096 rejections the walk ends, so a walk that starts on 0 -> 1 stops
    at length 2 with probability (1 - 1e-3)^4096."""
    from scipy.stats import binomtest
    o = O.Oracle(window=0, directed=True)
    o.ingest([0, 1], [1, 0], [1, 2])
    o.set_node2vec(1000.0, 1.0)
    node, tsa, ln, _, _ = o.walks(40_000, 3, bias=4, seed=17)
    on01 = (node[:, 0] == 0) & (node[:, 1] == 1)
    assert on01.sum() > 15_000
    stops = int((ln[on01] == 2).sum())
    p_stop = (1 - 1e-3) ** O.N2V_MAX_TRIALS
    assert binomtest(stops, int(on01.sum()), p_stop).pvalue > 1e-3, (stops, on01.sum(), p_stop)
    assert (ln[~on01] == 2).all()  # 1 -> 0 at t 2 has no continuation
    with pytest.raises(ValueError):
        o.set_node2vec(0.0, 1.0)


# ------------------------------------------------ the agreement rule's bound
def _exact_x(u, n, bias, lam, mp):
    """x of the sampler in 80-digit arithmetic from the exact u."""
    u, n, lam = mp.mpf(u), mp.mpf(n), mp.mpf(lam)
    if bias == 0:
        return u * n
    if bias == 1:
        return (mp.sqrt(1 + 4 * u * n * (n + 1)) - 1) / 2
    return n + mp.log(u + (1 - u) * mp.exp(-lam * n)) / lam


def _bound_cases(rng):
    ns = [1, 2, 7, 100, 10**4, 10**6, 1 << 24, 10**8, (1 << 31) - 1]
    for _ in range(4000):
        n = rng.choice(ns + [rng.randrange(1, 1 << 31)])
        lam = rng.choice([1.0, 3.0, 0.5, 1e-3, 1e-8, 1.0 / n, 30.0 / n])
        k = rng.choice([rng.randrange(1, 1 << 53), rng.randrange(1, 1 << 20), (1 << 53) - rng.randrange(1, 1 << 20)])
        yield k * 2.0 ** -53, n, lam


@pytest.mark.parametrize("bias", [0, 1, 2])
def test_double_evaluation_stays_within_its_bound(bias):
    """orc_sampler_x_bound bounds the rounding error of the oracle's own
    double evaluation of Eq. 1 / Eq. 2 / exact Eq. 3 against the value in
    80-digit arithmetic, for n up to 2^31 - 1, rates from 1e-8 to 30, and u
    near 0, near 1 and in between; the error reaches a visible share of the
    bound (it is not vacuous)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 80
    rng = random.Random(300 + bias)
    worst = 0.0
    for u, n, lam in _bound_cases(rng):
        if bias != 2:
            lam = 1.0
        x = O.sampler_x(u, n, bias, lam)
        b = O.sampler_x_bound(u, n, bias, lam)
        err = abs(mp.mpf(x) - _exact_x(u, n, bias, lam, mp))
        assert err <= b, (bias, u, n, lam, float(err), b)
        worst = max(worst, float(err / b))
    assert worst > 0.02


def test_exponential_bound_needs_its_rate_term():
    """A bound without the term in 1/lambda (the error of s carried through
    log(s) / lambda) is broken at small rates: the planted omission fails
    the same comparison, so the test above can see a dropped term."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 80
    rng = random.Random(77)
    eps = 2.0 ** -53
    broken = 0
    for _ in range(3000):
        n = rng.choice([10**4, 10**6, 10**8])
        lam = rng.choice([1e-8, 1e-3 / n, 1.0 / n])
        u = rng.randrange(1, 1 << 53) * 2.0 ** -53
        x = O.sampler_x(u, n, 2, lam)
        planted = eps * (2 * abs(x) + 6 * abs(x - n))
        if abs(mp.mpf(x) - _exact_x(u, n, 2, lam, mp)) > planted:
            broken += 1
    assert broken > 30


def test_agreement_margin_units():
    """sampler_batch's margin is |x - round(x)| / bound: zero on an exact
    boundary (linear u = 1/3 at n = 2 gives x = 1), large far from one."""
    k = np.array([int(round(2.0 ** 53 / 3)), 1 << 52], dtype=np.uint64)
    idx, mg = O.sampler_batch(k, np.array([2, 2], np.int64), 1)
    x = O.sampler_x(float(k[0]) * 2.0 ** -53, 2, 1)
    assert mg[0] == pytest.approx(abs(x - round(x)) / O.sampler_x_bound(float(k[0]) * 2.0 ** -53, 2, 1))
    assert mg[1] > 1e10  # u = 1/2: x = 1.3028, far from an integer
