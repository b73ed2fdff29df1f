"""The allocation-free batch sort (tempest_sort_batch_noalloc).

It serves callers that cannot allocate device memory at run time, so it uses
a fixed static scratch array instead.  The GPU test calls it through the C
ABI twice in a row -- the second call runs on whatever the first left in the
shared scratch -- and checks both results against the batch order the
regular ingest path produces (tempest_ingest into an unbounded window, then
the exported edge store) and against the oracle's live edges after the same
batch (a stable sort by timestamp, arrival order among ties).  Integer
results, so the comparison is exact.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_16182_gb300 import _lib


def _batch(rng, n, ts_lo, ts_hi):
    s = rng.integers(0, 1 << 30, n).astype(np.int32)
    d = rng.integers(0, 1 << 30, n).astype(np.int32)
    t = rng.integers(ts_lo, ts_hi, n).astype(np.int64)
    t[::7] = t[0]  # ties: arrival order must be kept
    return s, d, t


def _via_ingest(s, d, t):
    eng = _lib.Engine(window=0, directed=True, device="cuda:0")
    import torch
    eng.ingest(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(t).cuda())
    st = (eng.export(_lib.STATE_SRC), eng.export(_lib.STATE_DST), eng.export(_lib.STATE_TS))
    eng.close()
    return st


def _via_noalloc(s, d, t):
    import torch
    n = s.shape[0]
    src, dst, ts = (torch.from_numpy(x).cuda() for x in (s, d, t))
    o_s = torch.empty(n, dtype=torch.int32, device="cuda")
    o_d = torch.empty(n, dtype=torch.int32, device="cuda")
    o_t = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    _lib.tempest_sort_batch_noalloc(src.data_ptr(), dst.data_ptr(), ts.data_ptr(), n, o_s.data_ptr(),
                                    o_d.data_ptr(), o_t.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return o_s.cpu().numpy(), o_d.cpu().numpy(), o_t.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_sort_matches_ingest_on_two_calls_in_a_row():
    rng = np.random.default_rng(2024)
    batches = [_batch(rng, _lib.NOALLOC_MAX_EDGES, -(1 << 62), 1 << 62),   # the maximum size
               _batch(rng, 77_777, 0, 1000)]                                # smaller, many ties
    for s, d, t in batches:
        got = _via_noalloc(s, d, t)
        want = _via_ingest(s, d, t)
        orc = O.Oracle(0, True)
        orc.ingest(s, d, t)
        st = orc.state()
        orc.close()
        for g, w, o, name in zip(got, want, (st["src"], st["dst"], st["ts"]), ("src", "dst", "ts")):
            assert np.array_equal(g, w), name + " (ingest)"
            assert np.array_equal(g, o), name + " (oracle)"


def test_noalloc_rejects_oversized_batch():
    L = _lib.load()
    rc = L.tempest_sort_batch_noalloc(None, None, None, _lib.NOALLOC_MAX_EDGES + 1, None, None, None, None)
    assert rc == _lib.TEMPEST_EINVAL
    assert "maximum" in _lib.tempest_last_error(None)
    assert L.tempest_sort_batch_noalloc(None, None, None, -1, None, None, None, None) == _lib.TEMPEST_EINVAL
    assert L.tempest_sort_batch_noalloc(None, None, None, 0, None, None, None, None) == _lib.TEMPEST_OK
