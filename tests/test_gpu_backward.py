"""Backward walks (Sec. 2.1: the backward case defined analogously to the
forward one) on the GPU against the oracle, element by element.

A backward walk is a forward walk on the time-reversed graph, which holds
every live edge (u, v, t) as (v, u, -t) in mirrored arrival order: from node v
at time t it draws an in-edge of v earlier than t, latest first.  Directed
graphs read a second (in-edge) index that every ingest keeps once
tempest_enable_backward was called; undirected graphs walk their one view.
Uniform and linear walks must be bit-exact; exponential walks must agree on
>= 99.99 % of hops with every divergence at a sampler boundary.
"""
import random

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_16182_gb300 import _lib, synth
from parity_util import MIN_HOP_AGREEMENT, assert_walks_bit_exact, compare_biased

pytestmark = pytest.mark.gpu

SCHEDULERS = (_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_COOP, _lib.SCHED_GRAPH, _lib.SCHED_LANE)


def pair(window, directed, enable=True):
    eng = _lib.Engine(window=window, directed=directed, device="cuda:0")
    if enable:
        eng.enable_backward()
    return eng, O.Oracle(window, directed)


def ingest_both(eng, orc, s, d, t):
    s = np.ascontiguousarray(np.asarray(s), np.int32)
    d = np.ascontiguousarray(np.asarray(d), np.int32)
    t = np.ascontiguousarray(np.asarray(t), np.int64)
    eng.ingest(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(t).cuda())
    orc.ingest(s, d, t)


def check_back(eng, orc, n, L, policy=0, seed=0, biases=(0, 1, 2), scheds=SCHEDULERS):
    for sched in scheds:
        eng.set_scheduler(sched)
        for bias in biases:
            g = tuple(x.cpu().numpy() for x in eng.walks(n, L, bias=bias, start_policy=policy, seed=seed,
                                                         direction=1))
            o = orc.walks(n, L, bias=bias, start_policy=policy, seed=seed, with_margin=bias >= 2, direction=1)
            where = "backward sched %d bias %d policy %d" % (sched, bias, policy)
            if bias >= 2:
                agree, total, _ = compare_biased(g, o, o[3])
                assert total == 0 or agree / total >= MIN_HOP_AGREEMENT, (where, agree, total)
            else:
                assert_walks_bit_exact(g, o, where)
    eng.set_scheduler(_lib.SCHED_LANE)


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
@pytest.mark.parametrize("window", [0, 40, -25])
def test_random_streams_backward(directed, window):
    """Small random streams (ties, late batches, both window kinds): every
    walk form, every bias 0-2, both edge start policies."""
    rng = random.Random(77 + window * 5 + directed)
    for trial in range(5):
        eng, orc = pair(window, directed)
        for s, d, t in _stream(rng, rng.randrange(1, 6), rng.choice([5, 60, 700]),
                               rng.choice([1, 3, 50, 2000]), 100, rng.random() < 0.5):
            ingest_both(eng, orc, s, d, t)
        check_back(eng, orc, 600, rng.choice([2, 3, 9]), policy=trial % 2, seed=trial)


@pytest.mark.parametrize("directed", [1, 0])
def test_backward_streaming_hubs_all_forms(directed):
    """A stream with hubs, ties and window eviction, several tiles of walks;
    the in-edge index follows every batch."""
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, directed)
    for i, (_, s, d, t) in enumerate(spec.batches(last=7)):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
        if i in (0, 4, 6):
            check_back(eng, orc, 3000, 14, seed=40 + i, biases=(0, 2),
                       scheds=(_lib.SCHED_STREAM, _lib.SCHED_FULL_WALK, _lib.SCHED_LANE) if i < 6 else SCHEDULERS)
    check_back(eng, orc, 3000, 10, policy=_lib.START_BIASED_TS, seed=3, scheds=(_lib.SCHED_STREAM, _lib.SCHED_LANE))


def test_enable_backward_mid_stream_replays_the_live_edges():
    """Turned on after evictions and out-of-order merges, the in-edge index
    is built from the live edges alone and then follows later batches."""
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, 1, enable=False)
    batches = list(spec.batches(last=8))
    for _, s, d, t in batches[:5]:
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    with pytest.raises(_lib.TempestError) as e:
        eng.walks(10, 5, direction=1)
    assert e.value.code == _lib.TEMPEST_EINVAL
    eng.enable_backward()
    eng.enable_backward()  # a second call keeps the index
    check_back(eng, orc, 2000, 12, seed=5, biases=(0, 1), scheds=(_lib.SCHED_STREAM, _lib.SCHED_LANE))
    # a late batch (timestamps inside the window but older than the newest)
    _, s, d, t = batches[5]
    t_late = t.numpy() - (int(t.numpy().max()) - int(t.numpy().min())) // 2
    ingest_both(eng, orc, s.numpy(), d.numpy(), t_late)
    for _, s, d, t in batches[6:]:
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    check_back(eng, orc, 2000, 12, seed=6, biases=(0, 2), scheds=(_lib.SCHED_STREAM, _lib.SCHED_COOP, _lib.SCHED_LANE))


@pytest.mark.parametrize("directed", [1, 0])
def test_backward_per_node_walks(directed):
    """PER_NODE backward walks start after every live edge at each node with a
    live in-edge, in id order."""
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, directed)
    for _, s, d, t in spec.batches(last=5):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    na = eng.active_nodes(direction=1)
    assert na == len(orc.active_nodes(1)) > 0
    if directed:
        assert na != eng.active_nodes()  # in- and out-active sets differ on this stream
    for K in (1, 2):
        check_back(eng, orc, K * na, 12, policy=_lib.START_PER_NODE, seed=K)
    with pytest.raises(_lib.TempestError) as e:
        eng.walks(na + 1, 8, start_policy=_lib.START_PER_NODE, direction=1)
    assert e.value.code == _lib.TEMPEST_EINVAL


def test_backward_rejects_weight_bias_and_keeps_forward_intact():
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, 1)
    for _, s, d, t in spec.batches(last=3):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    with pytest.raises(_lib.TempestError) as e:
        eng.walks(10, 5, bias=_lib.BIAS_EXP_WEIGHT, direction=1)
    assert e.value.code == _lib.TEMPEST_EINVAL
    # forward walks are untouched by the second index
    g = tuple(x.cpu().numpy() for x in eng.walks(2000, 10, bias=1, seed=9))
    assert_walks_bit_exact(g, orc.walks(2000, 10, bias=1, seed=9), "forward with backward on")


def test_mixed_directions_in_one_batch_and_in_the_server():
    """A batch of forward and backward requests gives each request's walks as
    if it ran alone; the server runs them in single-direction waves."""
    spec = synth.config_mid(scale=0.005)
    eng, orc = pair(spec.window, 1)
    for _, s, d, t in spec.batches(last=4):
        ingest_both(eng, orc, s.numpy(), d.numpy(), t.numpy())
    specs = [(700, 9, 0, 0, 11, 0), (900, 12, 1, 0, 12, 1), (500, 7, 2, 1, 13, 1), (400, 10, 1, 1, 14, 0)]

    def outs(n, L):
        return (torch.empty((n, L), dtype=torch.int32, device="cuda"),
                torch.empty((n, L), dtype=torch.int64, device="cuda"),
                torch.empty((n,), dtype=torch.int32, device="cuda"))

    bufs = [outs(n, L) for n, L, *_ in specs]
    reqs = [_lib.make_request(n, L, b, p, sd, *o, direction=dr) for (n, L, b, p, sd, dr), o in zip(specs, bufs)]
    _lib.tempest_walks_batch(eng.h, reqs)
    torch.cuda.synchronize()
    st = eng.last_walk_stats()
    assert st["launches"] == 2
    for (n, L, b, p, sd, dr), o in zip(specs, bufs):
        alone = eng.walks(n, L, bias=b, start_policy=p, seed=sd, direction=dr)
        assert all(torch.equal(x, y) for x, y in zip(alone, o)), (n, dr)
        if b < 2:
            ow = orc.walks(n, L, bias=b, start_policy=p, seed=sd, direction=dr)
            assert_walks_bit_exact(tuple(x.cpu().numpy() for x in o), ow, "batched dir %d" % dr)

    srv = _lib.Server(eng, arena_bytes=64 << 20, max_wave_walks=1 << 20)
    tickets = [srv.submit_walks(_lib.make_request(n, L, b, p, sd, direction=dr)) for n, L, b, p, sd, dr in specs]
    srv.drain()
    for (n, L, b, p, sd, dr), tk in zip(specs, tickets):
        assert srv.status(tk)[0] == srv.DONE
        node, ts, ln = srv.result(tk, n, L)
        alone = eng.walks(n, L, bias=b, start_policy=p, seed=sd, direction=dr)
        assert torch.equal(alone[0], node) and torch.equal(alone[1], ts) and torch.equal(alone[2], ln)
        srv.release(tk)
    assert srv.stats()["waves"] >= 3  # directions alternate 0, 1, 1, 0
    srv.close()
