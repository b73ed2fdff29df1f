"""Temporal Node2Vec walks (Sec. 2.5) on the GPU against the oracle.

Each hop draws proposals from the exponential sampler and accepts one with
probability beta(u, w) / beta_max (rejection sampling on a prev-independent
proposal); both sides take the same Philox draws and the same exact double
comparison, so walks agree hop by hop except where an exponential proposal
sits on a sampler boundary (the agreement rule of the exponential bias).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_16182_gb300 import _lib, synth
from parity_util import MIN_HOP_AGREEMENT, assert_walks_bit_exact, compare_biased

pytestmark = pytest.mark.gpu

SCHEDULERS = (_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_COOP, _lib.SCHED_GRAPH, _lib.SCHED_LANE)
N2V = _lib.BIAS_NODE2VEC


def pair(window, directed, p, q, backward=False):
    eng = _lib.Engine(window=window, directed=directed, device="cuda:0")
    orc = O.Oracle(window, directed)
    eng.set_node2vec(p, q)
    orc.set_node2vec(p, q)
    if backward:
        eng.enable_backward()
    return eng, orc


def ingest_both(eng, orc, s, d, t):
    s = np.ascontiguousarray(np.asarray(s), np.int32)
    d = np.ascontiguousarray(np.asarray(d), np.int32)
    t = np.ascontiguousarray(np.asarray(t), np.int64)
    eng.ingest(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(t).cuda())
    orc.ingest(s, d, t)


def check_n2v(eng, orc, n, L, policy=0, seed=0, direction=0, scheds=SCHEDULERS):
    for sched in scheds:
        eng.set_scheduler(sched)
        g = tuple(x.cpu().numpy() for x in eng.walks(n, L, bias=N2V, start_policy=policy, seed=seed,
                                                     direction=direction))
        o = orc.walks(n, L, bias=N2V, start_policy=policy, seed=seed, with_margin=True, direction=direction)
        agree, total, _ = compare_biased(g, o, o[3])
        assert total == 0 or agree / total >= MIN_HOP_AGREEMENT, (sched, agree, total)
    eng.set_scheduler(_lib.SCHED_LANE)


@pytest.mark.parametrize("directed", [1, 0])
@pytest.mark.parametrize("pq", [(0.25, 4.0), (4.0, 0.5)])
def test_node2vec_streaming_all_forms(directed, pq):
    """A stream with hubs, ties and eviction: after ingests the pair table
    follows the window, and every walk form gives the oracle's walks."""
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, directed, *pq)
    for i, (_, s, d, t) in enumerate(spec.batches(last=7)):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
        if i in (0, 3, 6):
            check_n2v(eng, orc, 3000, 12, seed=60 + i,
                      scheds=SCHEDULERS if i == 6 else (_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_LANE))
    check_n2v(eng, orc, 3000, 10, policy=_lib.START_BIASED_TS, seed=4, scheds=(_lib.SCHED_STREAM, _lib.SCHED_LANE))


@pytest.mark.parametrize("directed", [1, 0])
def test_node2vec_backward_and_per_node(directed):
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, directed, 0.5, 2.0, backward=True)
    for _, s, d, t in spec.batches(last=5):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    check_n2v(eng, orc, 3000, 12, seed=8, direction=1)
    na = eng.active_nodes()
    check_n2v(eng, orc, 2 * na, 10, policy=_lib.START_PER_NODE, seed=9,
              scheds=(_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_COOP, _lib.SCHED_LANE))
    nb = eng.active_nodes(direction=1)
    check_n2v(eng, orc, nb, 10, policy=_lib.START_PER_NODE, seed=10, direction=1, scheds=(_lib.SCHED_STREAM, _lib.SCHED_LANE))


def test_node2vec_pair_table_under_sliding_window_and_rebuilds():
    """Many small batches (the used-slot bound crosses half the table several
    times, forcing rebuilds), repeated pairs, eviction of every pair's last
    copy and a late batch (a merge, which rebuilds); walks stay the oracle's."""
    eng, orc = pair(-600, 1, 0.3, 3.0)
    rng = np.random.default_rng(21)
    t = 0
    for b in range(40):
        n = int(rng.integers(50, 200))
        s = rng.integers(0, 40, n).astype(np.int32)
        d = rng.integers(0, 40, n).astype(np.int32)
        ts = (t + np.sort(rng.integers(0, 50, n))).astype(np.int64)
        t = int(ts[-1])
        if b == 25:
            ts = ts - 120  # late: inside the window, older than the newest edges
        ingest_both(eng, orc, s, d, ts)
        if b % 8 == 7 or b == 25:
            check_n2v(eng, orc, 1500, 10, seed=b, scheds=(_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_LANE))


def test_node2vec_unit_parameters_equal_exponential_walks():
    """p = q = 1: every proposal is accepted at once, so Node2Vec walks are
    the exponential walks bit for bit (the plain walker form runs them)."""
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, 1, 1.0, 1.0)
    for _, s, d, t in spec.batches(last=3):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    for sched in SCHEDULERS:
        eng.set_scheduler(sched)
        a = [x.clone() for x in eng.walks(4000, 12, bias=N2V, seed=5)]
        b = eng.walks(4000, 12, bias=_lib.BIAS_EXP, seed=5)
        assert all(torch.equal(x, y) for x, y in zip(a, b)), sched


def test_node2vec_rejection_cap_and_counters():
    """The two-edge graph of the oracle's cap pin (a return accepted with
    probability 1e-3): the GPU ends the same walks after 4096 rejections, and
    its hop and sector-model counters equal the oracle's accounting."""
    eng, orc = pair(0, 1, 1000.0, 1.0)
    ingest_both(eng, orc, [0, 1], [1, 0], [1, 2])
    o = orc.walks(20_000, 3, bias=N2V, seed=17, with_bytes=True)
    for sched in SCHEDULERS:
        eng.set_scheduler(sched)
        g = tuple(x.cpu().numpy() for x in eng.walks(20_000, 3, bias=N2V, seed=17))
        assert_walks_bit_exact(g, o, "sched %d" % sched)  # one group per draw: no boundary
        ws = eng.last_walk_stats()
        assert ws["hops"] == int(np.clip(o[2] - 1, 0, None).sum())
        assert ws["model_bytes"] == int(o[4]), sched
    stops = int(((g[0][:, 0] == 0) & (g[2] == 2)).sum())
    assert stops > 0  # the cap is reached on this graph


def test_node2vec_counters_on_a_stream():
    spec = synth.config_small()
    eng, orc = pair(spec.window, 1, 0.5, 2.0)
    for _, s, d, t in spec.batches():
        ingest_both(eng, orc, s, d, t)
    o = orc.walks(5000, 12, bias=N2V, seed=2, with_margin=True, with_bytes=True)
    for sched in SCHEDULERS:
        eng.set_scheduler(sched)
        g = tuple(x.cpu().numpy() for x in eng.walks(5000, 12, bias=N2V, seed=2))
        ws = eng.last_walk_stats()
        same = all(np.array_equal(a, b) for a, b in zip(g, o[:3]))
        if same:
            assert ws["hops"] == int(np.clip(o[2] - 1, 0, None).sum())
            assert ws["model_bytes"] == int(o[4]), sched
        else:  # a boundary divergence moves a few hops
            agree, total, _ = compare_biased(g, o, o[3])
            assert agree / total >= MIN_HOP_AGREEMENT
            assert abs(ws["model_bytes"] - o[4]) <= 1e-3 * o[4]


def test_node2vec_in_mixed_and_batched_requests():
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, 1, 0.5, 2.0)
    for _, s, d, t in spec.batches(last=3):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    n = 3000
    lens = np.full(n, 10, np.int32)
    bias = np.array([4, 2, 0] * (n // 3), np.uint8)
    o = orc.walks(n, 10, max_len_arr=lens, bias_arr=bias, seed=1, with_margin=True)
    for host in (True, False):
        la = lens if host else torch.from_numpy(lens).cuda()
        ba = bias if host else torch.from_numpy(bias).cuda()
        g = [x.cpu().numpy() for x in eng.walks_mixed(la, ba, seed=1, max_len_cap=10)]
        eng.last_walk_stats()
        agree, total, _ = compare_biased(g, o, o[3])
        assert agree / total >= MIN_HOP_AGREEMENT, host
    alone = [x.clone() for x in eng.walks(1000, 9, bias=N2V, seed=3)]
    outs = (torch.empty((1000, 9), dtype=torch.int32, device="cuda"),
            torch.empty((1000, 9), dtype=torch.int64, device="cuda"),
            torch.empty((1000,), dtype=torch.int32, device="cuda"))
    outs2 = (torch.empty((700, 8), dtype=torch.int32, device="cuda"),
             torch.empty((700, 8), dtype=torch.int64, device="cuda"),
             torch.empty((700,), dtype=torch.int32, device="cuda"))
    _lib.tempest_walks_batch(eng.h, [_lib.make_request(700, 8, 1, 0, 4, *outs2),
                                     _lib.make_request(1000, 9, N2V, 0, 3, *outs)])
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(alone, outs))


def test_node2vec_parameter_checks():
    eng = _lib.Engine(window=0, directed=1, device="cuda:0")
    for p, q in ((0.0, 1.0), (1.0, 2e3), (float("nan"), 1.0)):
        with pytest.raises(_lib.TempestError) as e:
            eng.set_node2vec(p, q)
        assert e.value.code == _lib.TEMPEST_EINVAL
