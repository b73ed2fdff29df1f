"""Walks over high-degree nodes, whose hop search goes through time buckets.

A node with at least 32 timestamp groups gets a bucket table over its time
range; the bracket it gives must contain the first later group for every
time, so every walk form must still return the oracle's walks.  The cases
put walks on hub timelines with the patterns that stress the bucket map:
uniform spacing, dense clusters with ties, gaps of 1e9 to 1e18, timestamps
near the int64 extremes, and nodes with 31, 32 and 33 groups (the
threshold), then change the state by streaming ingest so the tables are
rebuilt.
"""
import numpy as np
import pytest
import torch

from paper_2605_16182_gb300 import _lib, synth
from test_gpu_parity import SCHEDULERS, check_walks, ingest_both, pair

pytestmark = pytest.mark.gpu


def _hub_edges(rng):
    src, dst, ts = [], [], []

    def add(s, d, t):
        src.extend(s)
        dst.extend(d)
        ts.extend(int(x) for x in t)

    # node 0: self loops on a timeline with every pattern, plus exits to 1..5
    parts = [1000 + 7 * np.arange(200),                           # uniform
             10**6 + rng.integers(0, 50, 500),                     # dense cluster with ties
             10**12 + 10**9 * np.arange(100),                      # wide gaps
             np.array([-(4 * 10**18), -(4 * 10**18) + 1, 4 * 10**18, 4 * 10**18 - 3]),  # extremes
             2 * 10**6 + np.cumsum(rng.integers(0, 3, 300))]       # steps of 0..2
    for p in parts:
        n = len(p)
        add([0] * n, list(np.where(rng.random(n) < 0.9, 0, rng.integers(1, 6, n))), p)
    # nodes 10, 11, 12 with 31, 32, 33 groups (self loops) and node 13 with
    # 40 groups whose times coincide with node 0's cluster
    for v, g in ((10, 31), (11, 32), (12, 33)):
        add([v] * g, [v] * g, 5000 + 11 * np.arange(g))
    add([13] * 40, [0] * 40, 10**6 + np.arange(40))
    # feeders: edges into the hubs at times inside their ranges
    n = 400
    add(list(rng.integers(20, 60, n)), list(rng.choice([0, 10, 11, 12, 13], n)),
        rng.choice(np.array(ts, dtype=np.int64), n) - rng.integers(-2, 3, n))
    order = rng.permutation(len(src))
    return (np.array(src, np.int32)[order], np.array(dst, np.int32)[order],
            np.array(ts, np.int64)[order])


@pytest.mark.parametrize("directed", [1, 0])
def test_hub_timelines_all_forms(directed):
    rng = np.random.default_rng(7 + directed)
    eng, orc = pair(0, directed)
    s, d, t = _hub_edges(rng)
    ingest_both(eng, orc, s, d, t)
    for seed in (1, 2):
        check_walks(eng, orc, 6000, 24, policy=0, seed=seed)
    check_walks(eng, orc, 4000, 12, policy=1, seed=3, biases=(0, 2))


def test_bucket_density_knob_keeps_walks():
    rng = np.random.default_rng(11)
    eng, orc = pair(0, 1)
    s, d, t = _hub_edges(rng)
    ingest_both(eng, orc, s, d, t)
    ref = [x.clone() for x in eng.walks(5000, 20, bias=1, seed=4)]
    for lg in (0, 1, 3, 5):
        eng.set_tuning(_lib.TUNE_BKT_LOG, lg)
        got = eng.walks(5000, 20, bias=1, seed=4)
        assert all(torch.equal(a, b) for a, b in zip(ref, got)), lg
    check_walks(eng, orc, 3000, 20, seed=5, biases=(0, 1), scheds=(_lib.SCHED_STREAM, _lib.SCHED_LANE))


def test_tables_follow_streaming_ingest():
    """Window eviction and appends change every hub's group range; each walk
    call after an ingest must see tables of the new state."""
    spec = synth.config_mid(scale=0.01)
    eng, orc = pair(spec.window, 1)
    for i, (_, s, d, t) in enumerate(spec.batches()):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
        if i in (0, 3, 7, 12, 19):
            check_walks(eng, orc, 3000, 16, seed=100 + i, biases=(0, 2),
                        scheds=(_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_LANE))


@pytest.mark.parametrize("directed", [1, 0])
def test_tables_carried_across_slides_moves_and_rebuilds(directed):
    """Walks after every batch of a sliding window in which two hubs keep
    gaining groups (their regions slide and move, shifting their group
    indices), a quiet batch (evictions only), a batch that extends a hub's
    last group (same timestamp), a time gap that empties thousands of
    buckets, and a late batch (a merge, which renumbers every group): each
    build carries the previous tables forward and must still bracket the
    first later group everywhere."""
    rng = np.random.default_rng(40 + directed)
    eng, orc = pair(-3000, directed)
    t = 0
    last_ts = 0
    for b in range(45):
        n = 300
        if b == 20:
            n = 0  # evictions only (count window keeps the newest 3000)
        hubs = rng.random(n) < 0.7
        s = np.where(hubs, rng.integers(0, 2, n), rng.integers(2, 400, n)).astype(np.int32)
        d = np.where(rng.random(n) < 0.5, rng.integers(0, 2, n), rng.integers(2, 400, n)).astype(np.int32)
        gaps = rng.integers(1, 5, n)
        if b == 30:
            gaps[n // 2] = 10**9  # a time gap inside the batch
        ts = (t + np.cumsum(gaps)).astype(np.int64)
        if b == 25:
            ts[: n // 3] = last_ts  # extends the hubs' last groups
            ts = np.sort(ts)
        if b == 36:
            ts = ts - 600  # late: inside the window, older than the newest edges
        if n:
            t = int(ts.max())
            last_ts = int(ts.max())
        ingest_both(eng, orc, s, d, ts)
        check_walks(eng, orc, 1500, 16, seed=b, biases=(0, 2),
                    scheds=(_lib.SCHED_LANE, _lib.SCHED_STREAM) if b % 5 else SCHEDULERS)
