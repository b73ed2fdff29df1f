"""CUDA library vs oracle, element by element, through the C ABI.

Index state after every batch and uniform / linear walks must be bit-exact;
exponential walks must agree on >= 99.99 % of hops with every divergence at
a sampler boundary (the CUDA and libm exp / log may differ in the last place).
"""
import json
import os
import random

import time

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_16182_gb300 import _lib, synth
from parity_util import (MIN_HOP_AGREEMENT, assert_state_equal, assert_walks_bit_exact,
                         compare_biased)

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def pair(window, directed):
    return _lib.Engine(window=window, directed=directed, device="cuda:0"), O.Oracle(window, directed)


def ingest_both(eng, orc, s, d, t, on_gpu=True):
    s = np.ascontiguousarray(np.asarray(s), np.int32)
    d = np.ascontiguousarray(np.asarray(d), np.int32)
    t = np.ascontiguousarray(np.asarray(t), np.int64)
    if on_gpu:
        st = eng.ingest(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(t).cuda())
    else:
        st = eng.ingest(s, d, t)
    orc.ingest(s, d, t)
    return st


SCHEDULERS = (_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_COOP, _lib.SCHED_GRAPH, _lib.SCHED_LANE)


def walks_both(eng, orc, n, L, bias, policy=0, seed=0, margin=False):
    g = eng.walks(n, L, bias=bias, start_policy=policy, seed=seed)
    torch.cuda.synchronize()
    g = tuple(x.cpu().numpy() for x in g)
    o = orc.walks(n, L, bias=bias, start_policy=policy, seed=seed, with_margin=margin)
    return g, o


def check_walks(eng, orc, n, L, policy=0, seed=0, biases=(0, 1, 2), scheds=SCHEDULERS):
    """Every walk form must give the oracle's walks."""
    for sched in scheds:
        eng.set_scheduler(sched)
        for bias in biases:
            g, o = walks_both(eng, orc, n, L, bias, policy, seed, margin=(bias >= 2))
            if bias >= 2:
                agree, total, div = compare_biased(g, o, o[3])
                assert total == 0 or agree / total >= MIN_HOP_AGREEMENT, (sched, agree, total)
            else:
                assert_walks_bit_exact(g, o, "sched %d bias %d" % (sched, bias))
    eng.set_scheduler(_lib.SCHED_LANE)


# ------------------------------------------------------------------ state
def test_hand_worked_fixture_state():
    fx = json.load(open(os.path.join(GOLDEN, "tiny_stream.json")))
    eng, orc = pair(fx["window"], fx["directed"])
    for b, want in zip(fx["batches"], fx["expected"]):
        ingest_both(eng, orc, b["src"], b["dst"], b["ts"])
        st = eng.state()
        assert_state_equal(st, orc.state())
        for k in ("src", "dst", "ts", "ts_group_off", "node_off", "node_order", "node_group_off", "node_gidx"):
            assert list(st[k]) == want[k], k


def _stream(rng, n_batches, max_batch, n_nodes, span, monotone):
    out, t = [], 0
    for _ in range(n_batches):
        k = rng.randrange(0, max_batch + 1)
        s = [rng.randrange(0, n_nodes) for _ in range(k)]
        d = [rng.randrange(0, n_nodes) for _ in range(k)]
        if monotone:
            ts = []
            for _ in range(k):
                t += rng.choice([0, 0, 1, 3])
                ts.append(t)
        else:
            ts = [t + rng.randrange(-span // 3, span) for _ in range(k)]
            t += span // 2
        out.append((s, d, ts))
    return out


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("window", [0, 40, -1, -25, -300])
def test_random_streams_state_and_walks(directed, window):
    rng = random.Random(1000 + window * 7 + directed)
    for trial in range(6):
        eng, orc = pair(window, directed)
        for s, d, t in _stream(rng, rng.randrange(1, 7), rng.choice([5, 60, 700]),
                               rng.choice([1, 3, 50, 2000]), 100, rng.random() < 0.5):
            ingest_both(eng, orc, s, d, t, on_gpu=rng.random() < 0.5)
            assert_state_equal(eng.state(), orc.state(), "trial %d" % trial)
        check_walks(eng, orc, 700, rng.choice([2, 3, 9]), policy=trial % 2, seed=trial)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("directed", [True, False])
def test_eviction_modes_agree(mode, directed):
    """Both ways of finding what each node lost to eviction (counting the
    evicted endpoints; each active node searching its own entries for the
    new store head), forced on streams where the other would be chosen:
    duration and count windows, sorted, unsorted and late batches, hubs and
    self-loops; state after every batch."""
    rng = random.Random(4400 + mode * 10 + directed)
    for trial, window in enumerate((-30, 40, -1, 7, -500)):
        eng, orc = pair(window, directed)
        eng.set_tuning(_lib.TUNE_EVICT, mode)
        assert eng.get_tuning(_lib.TUNE_EVICT) == mode
        for s, d, t in _stream(rng, rng.randrange(1, 7), rng.choice([6, 60, 900]),
                               rng.choice([3, 50, 2000]), 60, rng.random() < 0.5):
            ingest_both(eng, orc, s, d, t)
            assert_state_equal(eng.state(), orc.state(), "mode %d window %d" % (mode, window))
        check_walks(eng, orc, 500, 5, seed=trial, biases=(0,), scheds=(_lib.SCHED_LANE,))
    with pytest.raises(_lib.TempestError):
        eng.set_tuning(_lib.TUNE_EVICT, 3)


def test_multi_tile_unsorted_batch_with_ragged_tail():
    # spans several radix-sort tiles and scan chunks, not a multiple of any
    rng = np.random.default_rng(5)
    n = 3 * 2048 * 7 + 1234
    s = rng.integers(0, 40_000, n).astype(np.int32)
    d = rng.integers(0, 40_000, n).astype(np.int32)
    t = rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64)
    t[::17] = 12345  # many ties
    for directed in (True, False):
        eng, orc = pair(-(n // 3), directed)
        ingest_both(eng, orc, s, d, t)
        ingest_both(eng, orc, s[: n // 2], d[: n // 2], t[: n // 2] + (1 << 41))
        assert_state_equal(eng.state(), orc.state())
        check_walks(eng, orc, 5000, 7)


def test_late_edges_and_general_merge():
    eng, orc = pair(50, True)
    ingest_both(eng, orc, [0, 1, 2, 3], [1, 2, 3, 0], [100, 110, 120, 130])
    # overlaps the store (general merge), one late edge (ts < 80)
    st = ingest_both(eng, orc, [3, 2, 1, 0, 4], [0, 0, 0, 0, 0], [125, 79, 105, 140, 100])
    assert st["n_dropped_late"] == 1
    assert_state_equal(eng.state(), orc.state())
    # whole batch late
    st = ingest_both(eng, orc, [1, 1], [2, 2], [10, 20])
    assert st["n_dropped_late"] == 2
    assert_state_equal(eng.state(), orc.state())


@pytest.mark.parametrize("window", [20, -6])
@pytest.mark.parametrize("directed", [True, False])
def test_sorted_batches_with_late_prefix(window, directed):
    """Batches that arrive in timestamp order but start below the cut-off in
    force: their late edges are a prefix, which the window step (computed in
    the statistics' round trip) skips on the device; ties sit at the cut."""
    eng, orc = pair(window, directed)
    rng = np.random.default_rng(5 + abs(window))
    t0, late = 100, 0
    for b in range(8):
        n = int(rng.integers(5, 15))
        ts = np.sort(rng.integers(t0 - 40, t0 + 40, n)).astype(np.int64)
        ts[: n // 3] = ts[0]  # a tie group at the front
        s = rng.integers(0, 7, n)
        d = rng.integers(0, 7, n)
        st = ingest_both(eng, orc, s, d, ts)
        assert st["sorted_input"] == 1
        late += st["n_dropped_late"]
        assert_state_equal(eng.state(), orc.state(), "batch %d" % b)
        t0 += 30
    assert late > 0
    check_walks(eng, orc, 500, 6, seed=3, biases=(0, 1), scheds=(_lib.SCHED_LANE, _lib.SCHED_STREAM))


def test_small_config_state_and_walks():
    spec = synth.config_small()
    eng, orc = pair(spec.window, True)
    for k, s, d, t in spec.batches():
        st = ingest_both(eng, orc, s, d, t)
        assert st["sorted_input"] == 0
    assert_state_equal(eng.state(), orc.state())
    check_walks(eng, orc, 10_000, 20, policy=0, seed=0)
    check_walks(eng, orc, 10_000, 20, policy=1, seed=1)
    # the device hop counter and sector model match the oracle's accounting
    _, _, ln, _, nbytes = orc.walks(10_000, 20, bias=0, seed=0, with_bytes=True)
    for sched in SCHEDULERS:
        eng.set_scheduler(sched)
        eng.walks(10_000, 20, bias=0, seed=0)
        ws = eng.last_walk_stats()
        assert ws["hops"] == int(np.clip(ln - 1, 0, None).sum())
        assert ws["model_bytes"] == int(nbytes)


def test_mid_config_scaled_stream():
    spec = synth.config_mid(scale=0.02)   # 20 batches of 20k, window 100k
    eng, orc = pair(spec.window, True)
    for k, s, d, t in spec.batches():
        ingest_both(eng, orc, s, d, t)
        if k % 5 == 4:
            assert_state_equal(eng.state(), orc.state(), "batch %d" % k)
            n = 20_000
            bias = (np.arange(n) % 3).astype(np.uint8)
            L = (5 + np.arange(n) % 36).astype(np.int32)   # mixed lengths, cap 40
            o = orc.walks(n, 40, bias_arr=bias, max_len_arr=L, start_policy=O.START_BIASED_TS, seed=k,
                          with_margin=True)
            for sched in SCHEDULERS:
                eng.set_scheduler(sched)
                g = eng.walks_mixed(torch.from_numpy(L).cuda(), torch.from_numpy(bias).cuda(),
                                    start_policy=_lib.START_BIASED_TS, seed=k, max_len_cap=40)
                torch.cuda.synchronize()
                g = tuple(x.cpu().numpy() for x in g)
                agree, total, div = compare_biased(g, o, o[3])
                assert agree / total >= MIN_HOP_AGREEMENT
                lin_or_uni = bias != 2
                assert (g[0][lin_or_uni] == o[0][lin_or_uni]).all()
                assert (g[1][lin_or_uni] == o[1][lin_or_uni]).all()


@pytest.mark.parametrize("directed", [True, False])
def test_large_batches_state(directed):
    """Batches of 9M edges (18M index entries undirected): the flag scans and
    sorts then give each block more than one tile, which smaller tests never
    reach.  Sorted, sorted with a late prefix (the flags start off a 16-byte
    boundary), and shuffled; state after every batch."""
    n, w = 9_000_000, -12_000_000
    spec = synth.StreamSpec("large-batches", 200_000, 3 * n, 1.6, 99, n, mean_gaps=[3, 1], switch_every=n // 3,
                            window=w)
    eng, orc = pair(w, directed)
    rng = np.random.default_rng(17)
    cut = None
    for k, s, d, t in spec.batches():
        s, d, t = s.numpy(), d.numpy(), t.numpy()
        if k == 2:
            # seven edges below the cut-off in force lead the sorted batch
            t = t.copy()
            t[:7] = cut - 5 - np.arange(7)[::-1]
            st = ingest_both(eng, orc, s, d, t)
            assert st["sorted_input"] == 1 and st["n_dropped_late"] == 7
        elif k == 1:
            p_ = rng.permutation(len(t))
            st = ingest_both(eng, orc, s[p_], d[p_], t[p_])
            assert st["sorted_input"] == 0
        else:
            st = ingest_both(eng, orc, s, d, t)
            assert st["sorted_input"] == 1
        assert_state_equal(eng.state(), orc.state(), "batch %d" % k)
        cut = orc.counts()["cutoff"]
    check_walks(eng, orc, 20_000, 12, seed=4, biases=(0,), scheds=(_lib.SCHED_LANE,))


@pytest.mark.parametrize("share", [62, 0, 100, 37])
def test_host_and_device_outputs_agree(share):
    """Walks into host buffers (part padded on the device and copied whole,
    part sent as cells and expanded by host threads, split by the host-link
    share, with a band between them that either side takes) equal the
    device-output walks row for row, padding included."""
    spec = synth.config_small(scale=0.3)
    eng, orc = pair(0, False)
    for k, s, d, t in spec.batches():
        ingest_both(eng, orc, s, d, t, on_gpu=False)
    eng.set_tuning(_lib.TUNE_HOST_LINK_PCT, share)
    assert eng.get_tuning(_lib.TUNE_HOST_LINK_PCT) == share
    eng.set_tuning(_lib.TUNE_HOST_THREADS, {62: 0, 0: 1, 100: 0, 37: 5}[share])  # 0: the process's CPUs
    for n, L in ((3000, 9), (40_000, 13), (1, 5)):
        gd = eng.walks(n, L, bias=1, seed=11)
        torch.cuda.synchronize()
        node = np.full((n, L), 7, np.int32)
        ts = np.full((n, L), 7, np.int64)
        ln = np.full(n, 7, np.int32)
        t0 = time.perf_counter()
        _lib.tempest_walks(eng.h, n, L, 1, 0, 11, node.ctypes.data, ts.ctypes.data, ln.ctypes.data)
        call_ms = 1e3 * (time.perf_counter() - t0)
        assert np.array_equal(node, gd[0].cpu().numpy()) and np.array_equal(ts, gd[1].cpu().numpy())
        assert np.array_equal(ln, gd[2].cpu().numpy())
        ws = eng.last_walk_stats()
        nd = n * share // 100
        nb = 0 if 0 < nd < n else nd  # rows [nb, nd) go either way
        base = 4 * n + 8 * (n - nb) + 12 * int(ln[nb:].sum())
        whole, rest = divmod(ws["d2h_bytes"] - base, 12 * L)
        assert rest == 0 and nb <= whole <= nd, (ws["d2h_bytes"], base, nb, nd)
        # the call's host-visible phases: each measured, together within the call
        assert all(x >= 0 for x in ws["host_ms"]) and ws["host_ms"][0] > 0
        assert sum(ws["host_ms"]) <= call_ms
        if n == 3000:
            o = orc.walks(n, L, bias=1, seed=11)
            assert_walks_bit_exact((node, ts, ln), o)
    eng.walks(100, 5, bias=1, seed=3)  # device outputs: no phases
    assert eng.last_walk_stats()["host_ms"] == [0.0, 0.0, 0.0]
    with pytest.raises(_lib.TempestError):
        eng.set_tuning(_lib.TUNE_HOST_LINK_PCT, 101)


@pytest.mark.parametrize("cap", [2, 3, 7, 8, 9, 12, 16, 33, 41, 64])
def test_row_lengths_around_the_staged_cells(cap):
    """A time-ordered chain 0 -> 1 -> ... -> 40 gives walks of every length
    from 2 to 41 nodes (a walk from edge i runs to the chain's end), so rows
    end before, at and after the cells a walker keeps on chip, at row widths
    that are and are not multiples of 4; every form, device and host outputs,
    and a mixed request with per-walk caps must give the oracle's rows."""
    eng, orc = pair(0, True)
    K = 40
    ingest_both(eng, orc, np.arange(K), np.arange(1, K + 1), np.arange(1, K + 1))
    check_walks(eng, orc, 2000, cap, seed=cap, biases=(0, 1))
    o = orc.walks(2000, cap, bias=0, seed=cap)
    assert set(np.unique(o[2])) == set(range(2, min(cap, K + 1) + 1))
    node = np.full((2000, cap), 5, np.int32)
    ts = np.full((2000, cap), 5, np.int64)
    ln = np.full(2000, 5, np.int32)
    _lib.tempest_walks(eng.h, 2000, cap, 0, 0, cap, node.ctypes.data, ts.ctypes.data, ln.ctypes.data)
    assert_walks_bit_exact((node, ts, ln), o, "host outputs")
    if cap >= 3:
        lens = np.random.default_rng(cap).integers(2, cap + 1, 2000).astype(np.int32)
        bias = np.zeros(2000, np.uint8)
        om = orc.walks(2000, cap, max_len_arr=lens, bias_arr=bias, seed=cap + 1)
        for sched in (_lib.SCHED_LANE, _lib.SCHED_STREAM):
            eng.set_scheduler(sched)
            g = [x.cpu().numpy() for x in eng.walks_mixed(torch.from_numpy(lens).cuda(), torch.from_numpy(bias).cuda(),
                                                          seed=cap + 1, max_len_cap=cap)]
            assert_walks_bit_exact(g, om, "mixed, sched %d" % sched)
        eng.set_scheduler(_lib.SCHED_LANE)


# ------------------------------------------------------------------ edges
def test_empty_and_degenerate():
    eng, orc = pair(0, True)
    g, o = walks_both(eng, orc, 5, 4, 0)
    assert (g[2] == 0).all() and (g[0] == -1).all()
    ingest_both(eng, orc, [], [], [])
    assert_state_equal(eng.state(), orc.state())
    # single node, self loops with equal timestamps
    ingest_both(eng, orc, [0, 0, 0], [0, 0, 0], [7, 7, 7])
    assert_state_equal(eng.state(), orc.state())
    check_walks(eng, orc, 100, 5)
    # max_len == 2, zero walks
    check_walks(eng, orc, 50, 2)
    eng.walks(0, 5)
    # a large sparse id
    ingest_both(eng, orc, [5_000_000], [3], [9])
    assert_state_equal(eng.state(), orc.state())
    check_walks(eng, orc, 300, 6)


def test_invalid_input_leaves_state_unchanged():
    eng, orc = pair(-5, True)
    ingest_both(eng, orc, [0, 1], [1, 0], [1, 2])
    before = eng.state()
    with pytest.raises(_lib.TempestError) as e:
        eng.ingest(torch.tensor([0, -3], dtype=torch.int32).cuda(), torch.tensor([1, 1], dtype=torch.int32).cuda(),
                   torch.tensor([5, 6], dtype=torch.int64).cuda())
    with pytest.raises(TypeError):
        eng.ingest(torch.tensor([0, 1]).cuda(), torch.tensor([1, 1]).cuda(), torch.tensor([5, 6]).cuda())
    assert e.value.code == _lib.TEMPEST_EINVAL
    assert_state_equal(eng.state(), before)
    with pytest.raises(_lib.TempestError):
        eng.walks(3, 1)
    with pytest.raises(_lib.TempestError):
        eng.walks(3, 4, bias=7)
    with pytest.raises(_lib.TempestError):
        eng.set_bias_params(0.0)


def test_bias_parameters():
    spec = synth.config_small(scale=0.1)
    eng, orc = pair(0, True)
    for k, s, d, t in spec.batches():
        ingest_both(eng, orc, s, d, t)
    for lh, ls in ((0.25, 0.0), (3.0, 1e-3)):
        eng.set_bias_params(lh, ls)
        orc.set_bias_params(lh, ls)
        check_walks(eng, orc, 4000, 8, policy=1, seed=4, biases=(2,))


def test_cooperative_tiers_are_all_exercised():
    """Per-hop regrouping (Alg. 1) reaches every tier of the dispatch plane on
    a hub-heavy graph, and its walks equal the oracle's."""
    rng = np.random.default_rng(9)
    eng, orc = pair(0, True)
    # a hub with many groups (block-global), a node with few groups and many
    # walks (block-smem / warp-smem), medium nodes and a long sparse tail
    n = 300_000
    s = np.where(rng.random(n) < 0.5, 0, rng.integers(1, 3000, n)).astype(np.int32)
    d = np.where(rng.random(n) < 0.5, 0, rng.integers(1, 3000, n)).astype(np.int32)
    t = rng.integers(0, 1_000_000, n).astype(np.int64)
    t[s == 7] = 5  # node 7: one group
    ingest_both(eng, orc, s, d, t)
    eng.set_scheduler(_lib.SCHED_COOP)
    for bias in (0, 2):
        g, o = walks_both(eng, orc, 200_000, 12, bias, 0, seed=3, margin=(bias == 2))
        if bias == 0:
            assert_walks_bit_exact(g, o)
        else:
            agree, total, _ = compare_biased(g, o, o[3])
            assert agree / total >= MIN_HOP_AGREEMENT
        tiers = eng.last_walk_stats()["tier_launches"]
        assert tiers[0] > 0 and tiers[4] > 0, tiers
    check_walks(eng, orc, 50_000, 30, policy=1, seed=8)


# ------------------------------------------------- index regions under growth
def test_growing_hub_moves_regions_and_rebuilds():
    """Without a window one node keeps growing: its regions move to larger
    ones every few batches and the pools run out (a full rebuild); every
    state array and the walks must stay the oracle's after every batch."""
    eng, orc = pair(0, 1)
    rng = np.random.default_rng(3)
    t = 0
    for b in range(14):
        n = 10 if b == 0 else int(rng.integers(200, 3000))
        s = np.where(rng.random(n) < 0.8, 0, rng.integers(1, 50 + 40 * b, n)).astype(np.int32)
        d = rng.integers(0, 60 + 40 * b, n).astype(np.int32)
        ts = (t + np.sort(rng.integers(0, 5 * n, n))).astype(np.int64)
        t = int(ts[-1])  # the next batch may start on the same timestamp
        ingest_both(eng, orc, s, d, ts)
        assert_state_equal(eng.state(), orc.state())
        if b % 4 == 3:
            check_walks(eng, orc, 2000, 12, seed=b, biases=(0, 1), scheds=(_lib.SCHED_STREAM, _lib.SCHED_LANE))


@pytest.mark.parametrize("directed", [1, 0])
def test_sliding_window_moves_store_and_regions(directed):
    """A count window over many small batches: the store's live range walks
    through its buffer and moves to the front of the other buffer, and node
    regions move as nodes drift; the state stays the oracle's throughout."""
    eng, orc = pair(-700, directed)
    rng = np.random.default_rng(5 + directed)
    t = 0
    timed = 0
    for b in range(40):
        n = int(rng.integers(0, 400))
        s = rng.integers(0, 30 + b, n).astype(np.int32)
        d = rng.integers(0, 30 + b, n).astype(np.int32)
        ts = (t + np.sort(rng.integers(0, 3 * n + 1, n))).astype(np.int64)
        if n:
            t = int(ts[-1])
        st = ingest_both(eng, orc, s, d, ts)
        assert_state_equal(eng.state(), orc.state())
        # the eviction's device time is reported when the batch evicted
        # edges (0 when none were, or when the batch rebuilt the node view)
        assert st["evict_ms"] >= 0.0
        if st["n_evicted"] == 0:
            assert st["evict_ms"] == 0.0
        timed += st["evict_ms"] > 0.0
    assert timed > 10
    check_walks(eng, orc, 3000, 16, seed=1, biases=(0, 2))


@pytest.mark.parametrize("window", [-700, -1500])
@pytest.mark.parametrize("directed", [1, 0])
def test_store_moves_with_copy_ahead(window, directed):
    """Many store moves: in the batches before its buffer fills, each batch
    copies a share of the live range to the other buffer, and the move then
    copies the rest.  Batch sizes vary (empty ones included), some batches
    arrive shuffled (merges, which write the other buffer and drop the copy
    made ahead), some carry edges below the cut-off; state after every
    batch."""
    eng, orc = pair(window, directed)
    eng.set_tuning(_lib.TUNE_MIRROR_MIN, 16)  # copy ahead from 16 live edges on
    rng = np.random.default_rng(31 + directed - window)
    t = 0
    for b in range(120):
        n = int(rng.integers(0, 500)) if b % 17 else 0
        s = rng.integers(0, 40, n).astype(np.int32)
        d = rng.integers(0, 40, n).astype(np.int32)
        ts = (t + np.sort(rng.integers(0, 2 * n + 1, n))).astype(np.int64)
        if n:
            t = int(ts[-1])
        if n and b % 11 == 5:
            ts = ts - int(rng.integers(0, 3 * n))  # some below the cut-off; arrival order kept
        if n and b % 13 == 7:
            p_ = rng.permutation(n)
            s, d, ts = s[p_], d[p_], ts[p_]
        ingest_both(eng, orc, s, d, ts)
        assert_state_equal(eng.state(), orc.state(), "batch %d" % b)
    check_walks(eng, orc, 2000, 12, seed=2, biases=(0,), scheds=(_lib.SCHED_LANE,))


@pytest.mark.parametrize("window", [-3000, -900])
@pytest.mark.parametrize("directed", [1, 0])
def test_big_nodes_copy_ahead_of_slides(window, directed):
    """A hub-dominated count window with the copy-ahead threshold at its
    minimum: in the batches before a big node's regions fill, each batch
    copies a share of the node's live range to their front and the batch
    that no longer fits moves the node onto the copy (or falls back to the
    whole slide); shuffled batches (merges) rebuild the view and drop every
    copy.  State after every batch; walks, weight-based included (weights
    copied before their group grew are recomputed)."""
    eng, orc = _weight_pair(window, directed, 1e-3)
    eng.set_tuning(_lib.TUNE_MIRROR_MIN, 16)
    assert eng.get_tuning(_lib.TUNE_MIRROR_MIN) == 16
    rng = np.random.default_rng(77 + directed - window)
    t = 0
    switched = 0
    for b in range(160):
        n = int(rng.integers(40, 360))
        hub = rng.random(n)
        s = np.where(hub < 0.6, 0, np.where(hub < 0.75, 1, rng.integers(2, 50, n))).astype(np.int32)
        d = np.where(rng.random(n) < 0.3, 0, rng.integers(1, 50, n)).astype(np.int32)
        ts = (t + np.sort(rng.integers(0, 2 * n, n))).astype(np.int64)
        t = int(ts[-1])
        if b % 53 == 40:
            p_ = rng.permutation(n)
            s, d, ts = s[p_], d[p_], ts[p_]
        st = ingest_both(eng, orc, s, d, ts)
        switched += st["copied_ahead"]
        assert_state_equal(eng.state(), orc.state(), "batch %d" % b)
        if b % 40 == 39:
            check_walks(eng, orc, 2000, 10, seed=b, biases=(0, 3), scheds=(_lib.SCHED_LANE,))
    assert switched >= 3  # the hub moved onto its copy made ahead more than once
    with pytest.raises(_lib.TempestError):
        eng.set_tuning(_lib.TUNE_MIRROR_MIN, 15)


# ------------------------------------------------------------ PER_NODE starts
@pytest.mark.parametrize("directed", [1, 0])
def test_per_node_walks_all_forms(directed):
    """K walks from every active node, in id order; bit-exact with the
    oracle for uniform and linear bias, the boundary rule for exponential,
    in every walk form, after streaming ingest with eviction."""
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, directed)
    for i, (_, s, d, t) in enumerate(spec.batches(last=6)):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    na = eng.active_nodes()
    assert na == len(orc.active_nodes()) > 0
    for K in (1, 3):
        check_walks(eng, orc, K * na, 12, policy=_lib.START_PER_NODE, seed=K)
    with pytest.raises(_lib.TempestError) as e:
        eng.walks(na + 1, 8, start_policy=_lib.START_PER_NODE)
    assert e.value.code == _lib.TEMPEST_EINVAL


def test_per_node_walks_in_a_batched_launch():
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, 1)
    for _, s, d, t in spec.batches(last=3):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    na = eng.active_nodes()
    alone = [x.clone() for x in eng.walks(2 * na, 10, bias=2, start_policy=_lib.START_PER_NODE, seed=4)]
    outs = (torch.empty((2 * na, 10), dtype=torch.int32, device="cuda"),
            torch.empty((2 * na, 10), dtype=torch.int64, device="cuda"),
            torch.empty((2 * na,), dtype=torch.int32, device="cuda"))
    outs2 = (torch.empty((500, 10), dtype=torch.int32, device="cuda"),
             torch.empty((500, 10), dtype=torch.int64, device="cuda"),
             torch.empty((500,), dtype=torch.int32, device="cuda"))
    other = _lib.make_request(500, 10, 0, 0, 7, *outs2)
    r = _lib.make_request(2 * na, 10, 2, _lib.START_PER_NODE, 4, *outs)
    _lib.tempest_walks_batch(eng.h, [other, r])
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(alone, outs))


@pytest.mark.parametrize("bad", [np.iinfo(np.int64).min, np.iinfo(np.int64).max])
def test_reserved_timestamps_are_rejected(bad):
    eng, orc = pair(0, 1)
    ingest_both(eng, orc, [0, 1], [1, 2], [5, 6])
    with pytest.raises(_lib.TempestError) as e:
        eng.ingest(torch.tensor([0, 3], dtype=torch.int32).cuda(), torch.tensor([1, 3], dtype=torch.int32).cuda(),
                   torch.tensor([7, bad], dtype=torch.int64).cuda())
    assert e.value.code == _lib.TEMPEST_EINVAL
    assert_state_equal(eng.state(), orc.state(), "state unchanged")



# ------------------------------------------------- weight-based sampler (Sec. 2.5)
def _weight_pair(window, directed, lam):
    eng, orc = pair(window, directed)
    eng.set_weight_rate(lam)
    orc.set_weight_rate(lam)
    return eng, orc


@pytest.mark.parametrize("directed", [1, 0])
def test_weight_based_walks_all_forms(directed):
    """Weight-based exponential walks (per-edge weights exp(lambda (t - t_min)))
    agree with the oracle in every walk form, under the boundary rule, on a
    stream with hubs, ties and eviction; the rate makes weights span e^0..e^30
    across a hub's window."""
    spec = synth.config_mid(scale=0.005)
    eng, orc = _weight_pair(spec.window, directed, 3e-6)
    for i, (_, s, d, t) in enumerate(spec.batches(last=7)):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
        if i in (0, 3, 6):
            check_walks(eng, orc, 4000, 14, seed=20 + i, biases=(3,))
    check_walks(eng, orc, 3000, 10, policy=_lib.START_BIASED_TS, seed=9, biases=(3,),
                scheds=(_lib.SCHED_STREAM, _lib.SCHED_LANE))


def test_weight_based_walks_after_reference_moves():
    """A rate so large that every batch pushes new groups' exponents past the
    rebase threshold: each node's reference moves and all weights are
    recomputed; walks stay the oracle's."""
    eng, orc = _weight_pair(-3000, 1, 0.05)
    rng = np.random.default_rng(8)
    t = 0
    for b in range(8):
        n = 1500
        s = np.where(rng.random(n) < 0.6, 0, rng.integers(1, 30, n)).astype(np.int32)
        d = np.where(rng.random(n) < 0.6, 0, rng.integers(1, 30, n)).astype(np.int32)
        ts = (t + np.sort(rng.integers(0, 20000, n))).astype(np.int64)
        t = int(ts[-1])
        ingest_both(eng, orc, s, d, ts)
        check_walks(eng, orc, 2000, 12, seed=b, biases=(3,), scheds=(_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_LANE))


def test_weight_bias_in_mixed_and_batched_requests():
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, 1)
    for _, s, d, t in spec.batches(last=3):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    n = 3000
    lens = torch.full((n,), 10, dtype=torch.int32).cuda()
    bias = torch.tensor([3, 2, 0] * (n // 3), dtype=torch.uint8).cuda()
    # device per-walk biases before the weights are kept: EINVAL, walks clamped
    eng.walks_mixed(lens, bias, seed=1, max_len_cap=10)
    with pytest.raises(_lib.TempestError) as e:
        eng.last_walk_stats()
    assert e.value.code == _lib.TEMPEST_EINVAL
    eng.set_weight_rate(1e-9)
    g = [x.cpu().numpy() for x in eng.walks_mixed(lens, bias, seed=1, max_len_cap=10)]
    eng.last_walk_stats()
    o = orc.walks(n, 10, max_len_arr=lens.cpu().numpy(), bias_arr=bias.cpu().numpy(), seed=1, with_margin=True)
    agree, total, _ = compare_biased(g, o, o[3])
    assert total == 0 or agree / total >= MIN_HOP_AGREEMENT
    # the same walks from a batched launch
    outs = (torch.empty((n, 10), dtype=torch.int32, device="cuda"),
            torch.empty((n, 10), dtype=torch.int64, device="cuda"),
            torch.empty((n,), dtype=torch.int32, device="cuda"))
    _lib.tempest_walks_batch(eng.h, [_lib.make_request(n, 10, 0, 0, 1, *outs, max_len_arr=lens, bias_arr=bias)])
    torch.cuda.synchronize()
    assert all(np.array_equal(a, b.cpu().numpy()) for a, b in zip(g, outs))
