"""Batched walk requests and the serving loop.

Every request must give the same walks alone (a plain tempest_walks call on
the same index state) and in a mix: in one tempest_walks_batch launch, or
through the server's waves with an ingest interleaved.  Alone and in the mix
both run the same device code, so the comparison is exact; one request is
also checked against the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_16182_gb300 import _lib, synth
from parity_util import MIN_HOP_AGREEMENT, compare_biased

pytestmark = pytest.mark.gpu


def _engine_with_stream(batches):
    spec = synth.config_mid(scale=0.01)   # 10k-edge batches, window 50k
    eng = _lib.Engine(window=spec.window, directed=True, device="cuda:0")
    orc = O.Oracle(spec.window, True)
    data = [(s.cuda(), d.cuda(), t.cuda(), s.numpy(), d.numpy(), t.numpy()) for _, s, d, t in spec.batches()]
    for s, d, t, sn, dn, tn in data[:batches]:
        eng.ingest(s, d, t)
        orc.ingest(sn, dn, tn)
    return eng, orc, data


def _mix(rng, n_req):
    reqs = []
    for i in range(n_req):
        n = int(rng.choice([1, 7, 100, 3000, 20000]))
        L = int(rng.integers(2, 40))
        mixed = rng.random() < 0.3
        reqs.append(dict(n=n, L=L, bias=int(rng.integers(0, 3)), policy=int(rng.integers(0, 2)),
                         seed=int(rng.integers(0, 1 << 62)), mixed=mixed,
                         Larr=torch.from_numpy(rng.integers(2, L + 1, n).astype(np.int32)).cuda() if mixed else None,
                         barr=torch.from_numpy(rng.integers(0, 3, n).astype(np.uint8)).cuda() if mixed else None))
    return reqs


def _alone(eng, q):
    if q["mixed"]:
        return eng.walks_mixed(q["Larr"], q["barr"], start_policy=q["policy"], seed=q["seed"], max_len_cap=q["L"])
    return eng.walks(q["n"], q["L"], bias=q["bias"], start_policy=q["policy"], seed=q["seed"])


def _request(q, with_outputs):
    outs = (None, None, None)
    if with_outputs:
        outs = (torch.empty((q["n"], q["L"]), dtype=torch.int32, device="cuda"),
                torch.empty((q["n"], q["L"]), dtype=torch.int64, device="cuda"),
                torch.empty((q["n"],), dtype=torch.int32, device="cuda"))
    r = _lib.make_request(q["n"], q["L"], q["bias"], q["policy"], q["seed"], *outs,
                          max_len_arr=q["Larr"], bias_arr=q["barr"])
    return r, outs


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


def test_batch_launch_equals_requests_alone():
    eng, orc, _ = _engine_with_stream(6)
    rng = np.random.default_rng(1)
    mix = _mix(rng, 12)
    alone = [tuple(x.clone() for x in _alone(eng, q)) for q in mix]
    reqs, outs = zip(*[_request(q, True) for q in mix])
    _lib.tempest_walks_batch(eng.h, list(reqs))
    torch.cuda.synchronize()
    for q, a, o in zip(mix, alone, outs):
        assert _same(a, o), q
    # one request against the oracle as well
    q = next(q for q in mix if not q["mixed"] and q["n"] >= 100)
    node, ts, ln = (x.cpu().numpy() for x in alone[mix.index(q)])
    o = orc.walks(q["n"], q["L"], bias=q["bias"], start_policy=q["policy"], seed=q["seed"], with_margin=True)
    agree, total, _ = compare_biased((node, ts, ln), o, o[3])
    assert total == 0 or agree / total >= MIN_HOP_AGREEMENT


def test_server_waves_and_interleaved_ingest():
    eng, orc, data = _engine_with_stream(5)
    rng = np.random.default_rng(2)
    before, after = _mix(rng, 10), _mix(rng, 10)
    alone_before = [tuple(x.clone() for x in _alone(eng, q)) for q in before]
    srv = _lib.Server(eng, arena_bytes=1 << 30, max_wave_walks=30_000, max_inflight=2)
    tickets = []
    for i, q in enumerate(before):
        r, outs = _request(q, with_outputs=(i % 2 == 0))
        tickets.append((srv.submit_walks(r), q, outs))
        srv.progress()
    s, d, t = data[5][:3]
    srv.submit_ingest(s, d, t)             # epoch barrier
    tickets_after = []
    for i, q in enumerate(after):
        r, outs = _request(q, with_outputs=(i % 2 == 1))
        tickets_after.append((srv.submit_walks(r), q, outs))
    srv.drain()
    st = srv.stats()
    assert st["ingests"] == 1 and st["queued"] == 0 and st["waves"] >= 2
    torch.cuda.synchronize()
    for (tk, q, outs), a in zip(tickets, alone_before):
        state, _, lat = srv.status(tk)
        assert state == srv.DONE and lat >= 0
        got = outs if outs[0] is not None else srv.result(tk, q["n"], q["L"])
        assert _same(a, got), q
        srv.release(tk)
    # the ingest ran after every earlier request: later requests see the new state
    ref = _lib.Engine(window=synth.config_mid(scale=0.01).window, directed=True, device="cuda:0")
    for s2, d2, t2 in [x[:3] for x in data[:6]]:
        ref.ingest(s2, d2, t2)
    for tk, q, outs in tickets_after:
        got = outs if outs[0] is not None else srv.result(tk, q["n"], q["L"])
        assert _same(_alone(ref, q), got), q
        srv.release(tk)
    srv.close()


def test_server_admission_by_output_memory():
    eng, _, _ = _engine_with_stream(3)
    q = dict(n=4000, L=20, bias=0, policy=0, seed=5, mixed=False, Larr=None, barr=None)
    one = 4000 * 20 * 12 + 4000 * 4 + 1024
    srv = _lib.Server(eng, arena_bytes=one + one // 2, max_wave_walks=1_000_000, max_inflight=2)
    t1 = srv.submit_walks(_request(q, False)[0])
    t2 = srv.submit_walks(_request(dict(q, seed=6), False)[0])
    big = srv.submit_walks(_request(dict(q, n=40_000), False)[0])   # can never fit
    for _ in range(200):
        srv.progress()
        torch.cuda.synchronize()
    assert srv.status(t1)[0] == srv.DONE
    assert srv.status(t2)[0] == srv.QUEUED      # waits for memory held by t1
    srv.release(t1)
    srv.drain()
    assert srv.status(t2)[0] == srv.DONE
    assert srv.status(big)[0] == _lib.TEMPEST_ENOMEM
    a = _alone(eng, dict(q, seed=6))
    assert _same(a, srv.result(t2, 4000, 20))
    srv.close()
