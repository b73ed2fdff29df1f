"""Failure handling through the C ABI, injected on the host (no GPU fault).

An allocator callback that returns NULL stands in for device memory running
out, and an HBM budget below the next batch's need for a budget that is
spent.  A failed ingest must return ENOMEM and change nothing: the exported
state stays the oracle's state before the batch, the batch can be ingested
again once memory is back, and the stream then ends in the oracle's state
with the oracle's walks.  A failed walk call changes no state either.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_16182_gb300 import _lib, synth
from parity_util import assert_state_equal, assert_walks_bit_exact

pytestmark = pytest.mark.gpu


class FaultyAllocator:
    """Device memory from PyTorch's caching allocator; after arm(j) the j-th
    request from then on (and, with persist, every later one) returns NULL."""

    def __init__(self, stream):
        self.stream = stream
        self.count = 0
        self.fail_at = None
        self.persist = False
        self.failed = 0
        self.live = {}
        self.peak = 0
        dev = torch.cuda.current_device()

        @_lib.ALLOC_FN
        def alloc(nbytes, ctx):
            i = self.count
            self.count += 1
            if self.fail_at is not None and (i == self.fail_at or (self.persist and i > self.fail_at)):
                self.failed += 1
                return None
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, self.stream)
            except Exception:
                return None
            self.live[p] = int(nbytes)
            self.peak = max(self.peak, sum(self.live.values()))
            return p

        @_lib.RELEASE_FN
        def release(ptr, ctx):
            self.live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

        self.fns = (alloc, release)

    def arm(self, j, persist=False):
        self.fail_at = self.count + j
        self.persist = persist
        self.failed = 0

    def disarm(self):
        self.fail_at = None
        self.persist = False


def engine(window, directed, backward=False, budget=0):
    eng = _lib.Engine(window=window, directed=directed, device="cuda:0")
    fa = FaultyAllocator(eng.stream)
    _lib.tempest_set_allocator(eng.h, fa.fns[0], fa.fns[1], None, budget)
    if backward:
        eng.enable_backward()
    return eng, fa


def stream_batches(n_batches=12, batch=4000, window=-12000):
    spec = synth.StreamSpec("failure-stream", 3000, n_batches * batch, 1.6, 4242, batch, mean_gaps=[1000, 50],
                            switch_every=batch, window=window)
    return spec, [(s.numpy(), d.numpy(), t.numpy()) for _, s, d, t in spec.batches()]


def oracle_states(spec, batches, directed):
    """The oracle's state after each batch (index 0: before the first)."""
    orc = O.Oracle(spec.window, directed)
    out = [orc.state()]
    for s, d, t in batches:
        orc.ingest(s, d, t)
        out.append(orc.state())
    return orc, out


def ingest(eng, b):
    s, d, t = (torch.from_numpy(x).cuda() for x in b)
    return eng.ingest(s, d, t)


def alloc_counts(spec, batches, directed, backward, rebuilt=None):
    """Allocations each batch's ingest makes on a clean run (and, into the
    list rebuilt, whether it rebuilt the node view whole)."""
    eng, fa = engine(spec.window, directed, backward)
    counts = []
    for b in batches:
        c0 = fa.count
        st = ingest(eng, b)
        counts.append(fa.count - c0)
        if rebuilt is not None:
            rebuilt.append(st["view_rebuilt"])
    eng.close()
    return counts


def check_walks_equal(eng, orc, direction=0):
    g = eng.walks(3000, 10, bias=_lib.BIAS_UNIFORM, seed=5, direction=direction)
    torch.cuda.synchronize()
    o = orc.walks(3000, 10, bias=O.BIAS_UNIFORM, seed=5, direction=direction)
    assert_walks_bit_exact(tuple(x.cpu().numpy() for x in g), o[:3], "walks after the failures")


@pytest.mark.parametrize("directed,backward", [(True, False), (False, False), (True, True)])
def test_failed_allocation_in_ingest_changes_nothing(directed, backward):
    """Every allocation an ingest makes, failed in turn: ENOMEM, the state of
    before the batch, and the stream continues to the oracle's end state."""
    spec, batches = stream_batches()
    orc, states = oracle_states(spec, batches, directed)
    counts = alloc_counts(spec, batches, directed, backward)
    cases = [(k, j) for k, c in enumerate(counts) for j in range(c)]
    assert len(cases) >= 10, counts  # the stream grows its buffers in many places
    step = max(1, len(cases) // 40)
    for k, j in cases[::step]:
        eng, fa = engine(spec.window, directed, backward)
        for b in batches[:k]:
            ingest(eng, b)
        fa.arm(j)
        with pytest.raises(_lib.TempestError) as ei:
            ingest(eng, batches[k])
        assert ei.value.code == _lib.TEMPEST_ENOMEM, (k, j, str(ei.value))
        assert fa.failed == 1
        fa.disarm()
        assert_state_equal(eng.state(), states[k], "batch %d, allocation %d failed" % (k, j))
        for b in batches[k:]:
            ingest(eng, b)
        assert_state_equal(eng.state(), states[-1], "end of stream after batch %d failed once" % k)
        eng.close()
    check_walks_equal_end(spec, batches, orc, directed, backward)


def check_walks_equal_end(spec, batches, orc, directed, backward):
    eng, fa = engine(spec.window, directed, backward)
    for b in batches:
        ingest(eng, b)
    check_walks_equal(eng, orc)
    if backward:
        check_walks_equal(eng, orc, direction=1)
    eng.close()


@pytest.mark.parametrize("directed", [True, False])
def test_memory_that_stays_short_is_repaired_later(directed):
    """Every allocation from the j-th on fails: the ingest returns ENOMEM and
    its counters are those of before the batch; a call that must rebuild the
    views while memory stays short returns ENOMEM too, or, when the rebuild
    found its buffers in place, the state of before the batch; once memory
    is back the state is the one before the batch."""
    spec, batches = stream_batches()
    _, states = oracle_states(spec, batches, directed)
    counts = alloc_counts(spec, batches, directed, False)
    k = next(i for i, c in enumerate(counts) if i >= 3 and c >= 2)
    for j in range(counts[k]):
        eng, fa = engine(spec.window, directed)
        for b in batches[:k]:
            ingest(eng, b)
        fa.arm(j, persist=True)
        with pytest.raises(_lib.TempestError) as ei:
            ingest(eng, batches[k])
        assert ei.value.code == _lib.TEMPEST_ENOMEM
        c = eng.counts()
        for key in ("m", "G_tot", "n_nodes", "M", "Gn", "dropped_late", "evicted", "seq_next"):
            assert c[key] == states[k]["counts"][key], (k, j, key)
        try:
            assert_state_equal(eng.state(), states[k], "memory still short")
        except _lib.TempestError as e:
            assert e.code == _lib.TEMPEST_ENOMEM, str(e)
        fa.disarm()
        assert_state_equal(eng.state(), states[k], "batch %d, allocations from %d on failed" % (k, j))
        for b in batches[k:]:
            ingest(eng, b)
        assert_state_equal(eng.state(), states[-1], "end of stream")
        eng.close()


def test_hbm_budget_below_the_next_batch():
    """A budget set just above what the handle holds, before an appending
    batch that needs more: that ingest returns ENOMEM (the budget's message)
    before it changes anything, so the state of before the batch reads out
    under the same budget; with the budget lifted (same allocator) the same
    batch goes in and the stream ends in the oracle's state."""
    spec, batches = stream_batches()
    _, states = oracle_states(spec, batches, True)
    rebuilt = []
    counts = alloc_counts(spec, batches, True, False, rebuilt)
    k = next(i for i, c in enumerate(counts) if i >= 2 and c > 0 and not rebuilt[i])
    eng, fa = engine(spec.window, True)
    for b in batches[:k]:
        ingest(eng, b)
    # one read-out first: it sizes the export's staging buffer, which a
    # read-out of the same state under the budget then finds in place
    assert_state_equal(eng.state(), states[k], "before the budget")
    held = sum(fa.live.values())
    _lib.tempest_set_allocator(eng.h, fa.fns[0], fa.fns[1], None, held + 256)
    with pytest.raises(_lib.TempestError) as ei:
        ingest(eng, batches[k])
    assert ei.value.code == _lib.TEMPEST_ENOMEM and "budget" in str(ei.value), str(ei.value)
    assert sum(fa.live.values()) <= held + 256
    assert_state_equal(eng.state(), states[k], "budget reached at batch %d" % k)
    _lib.tempest_set_allocator(eng.h, fa.fns[0], fa.fns[1], None, 0)
    for b in batches[k:]:
        ingest(eng, b)
    assert_state_equal(eng.state(), states[-1], "end of stream after the budget was lifted")
    eng.close()


@pytest.mark.parametrize("sched", [_lib.SCHED_LANE, _lib.SCHED_COOP])
def test_failed_allocation_in_walk_call_changes_nothing(sched):
    """Each allocation of a walk call's first run on a new state, failed in
    turn: ENOMEM, the index unchanged, and the next call gives the oracle's
    walks."""
    spec, batches = stream_batches()
    orc, states = oracle_states(spec, batches, True)

    def fresh():
        eng, fa = engine(spec.window, True)
        eng.set_scheduler(sched)
        for b in batches:
            ingest(eng, b)
        return eng, fa

    eng, fa = fresh()
    c0 = fa.count
    check_walks_equal(eng, orc)
    n_alloc = fa.count - c0
    eng.close()
    assert n_alloc >= 2  # walk counters, bucket tables (the hub has >= 32 groups), scheduler buffers
    for j in range(n_alloc):
        eng, fa = fresh()
        fa.arm(j)
        with pytest.raises(_lib.TempestError) as ei:
            eng.walks(3000, 10, bias=_lib.BIAS_UNIFORM, seed=5)
        assert ei.value.code == _lib.TEMPEST_ENOMEM, str(ei.value)
        assert fa.failed == 1
        fa.disarm()
        assert_state_equal(eng.state(), states[-1], "walk allocation %d failed" % j)
        check_walks_equal(eng, orc)
        eng.close()


def test_failed_ingest_keeps_the_node2vec_pair_table():
    """With Temporal Node2Vec on, ingest keeps the live-pair table: a failed
    ingest restores it with the store, and the walks after the stream agree
    with the oracle's."""
    from parity_util import MIN_HOP_AGREEMENT, compare_biased
    spec, batches = stream_batches()
    orc, states = oracle_states(spec, batches, True)
    orc.set_node2vec(0.5, 2.0)
    eng, fa = engine(spec.window, True)
    eng.set_node2vec(0.5, 2.0)
    # the batches whose ingest allocates (the pair table grows with the window)
    ceng, cfa = engine(spec.window, True)
    ceng.set_node2vec(0.5, 2.0)
    grow = []
    for k, b in enumerate(batches):
        c0 = cfa.count
        ingest(ceng, b)
        if cfa.count > c0 and k >= 1:
            grow.append(k)
    ceng.close()
    assert len(grow) >= 2, grow
    for k, b in enumerate(batches):
        if k in grow[:2]:
            fa.arm(0, persist=True)
            with pytest.raises(_lib.TempestError):
                ingest(eng, b)
            fa.disarm()
            assert_state_equal(eng.state(), states[k], "node2vec, batch %d" % k)
        ingest(eng, b)
    g = eng.walks(3000, 10, bias=_lib.BIAS_NODE2VEC, seed=9)
    torch.cuda.synchronize()
    g = tuple(x.cpu().numpy() for x in g)
    o = orc.walks(3000, 10, bias=O.BIAS_NODE2VEC, seed=9, with_margin=True)
    agree, total, _ = compare_biased(g, o, o[3])
    assert total > 0 and agree / total >= MIN_HOP_AGREEMENT
    eng.close()


def test_destroy_returns_every_allocation():
    """After a stream with appends, evictions, rebuilds, walks in every form
    and the weight and in-edge indexes, destroying the handle hands every
    buffer it took from the allocator back to it."""
    spec, batches = stream_batches()
    eng, fa = engine(spec.window, True, backward=True)
    eng.set_weight_rate(1e-3)
    for b in batches:
        ingest(eng, b)
    for sched in (_lib.SCHED_LANE, _lib.SCHED_STREAM, _lib.SCHED_GRAPH, _lib.SCHED_COOP, _lib.SCHED_FULL_WALK):
        eng.set_scheduler(sched)
        eng.walks(2000, 8, bias=_lib.BIAS_EXP, seed=1)
    eng.walks(2000, 8, bias=_lib.BIAS_EXP_WEIGHT, seed=2)
    eng.walks(2000, 8, bias=_lib.BIAS_UNIFORM, seed=3, direction=1)
    # walks into host buffers (device staging for the rows and the cells)
    node, ts, ln = np.zeros((2000, 8), np.int32), np.zeros((2000, 8), np.int64), np.zeros(2000, np.int32)
    _lib.tempest_walks(eng.h, 2000, 8, 1, 0, 4, node.ctypes.data, ts.ctypes.data, ln.ctypes.data)
    torch.cuda.synchronize()
    assert fa.live
    eng.close()
    assert not fa.live, "%d buffers (%d bytes) still held after destroy" % (len(fa.live), sum(fa.live.values()))

