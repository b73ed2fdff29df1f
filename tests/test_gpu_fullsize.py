"""Full-size parity: the billion-edge stream's launch configuration, sampled.

The engine ingests 25 batches of 10M edges of the billion-edge stream (100M
node ids, Zipf 2.0, count window 200M edges) and draws 10M walks of max_len
80 in one call, in every walk form, as the benchmark does.  The oracle
ingests the same synthetic edges of the live window (the last 21 batches as
one batch: its count window keeps the newest 200M and the tie group at the
cut, the same live set as the engine's incremental eviction) and replays a
random sample of the walk ids one by one.  Uniform walks must be bit-exact;
exponential walks must agree on >= 99.99 % of hops with every divergence at a
sampler boundary.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_16182_gb300 import _lib, synth
from parity_util import MIN_HOP_AGREEMENT, assert_walks_bit_exact, compare_biased

pytestmark = pytest.mark.gpu

N_BATCHES = 25
N_WALKS = 10_000_000
MAX_LEN = 80
SAMPLE = 3000
FORMS = (_lib.SCHED_LANE, _lib.SCHED_STREAM, _lib.SCHED_GRAPH, _lib.SCHED_COOP, _lib.SCHED_FULL_WALK)


@pytest.fixture(scope="module")
def full_size():
    free, _ = torch.cuda.mem_get_info()
    if free < 120 << 30:
        pytest.skip("needs about 120 GB of free device memory")
    spec = synth.config_billion()
    eng = _lib.Engine(window=spec.window, directed=True, device="cuda:0")
    keep = N_BATCHES - (-spec.window) // spec.batch - 1  # first batch the oracle sees
    host = []
    for k, s, d, t in spec.batches(device="cuda", first=0, last=N_BATCHES):
        eng.ingest(s, d, t)
        if k >= keep:
            host.append((s.cpu().numpy(), d.cpu().numpy(), t.cpu().numpy()))
    torch.cuda.synchronize()
    assert eng.counts()["m"] >= -spec.window
    ids = np.sort(np.random.default_rng(77).choice(N_WALKS, SAMPLE, replace=False)).astype(np.int64)
    runs = {}
    out = (torch.empty((N_WALKS, MAX_LEN), dtype=torch.int32, device="cuda"),
           torch.empty((N_WALKS, MAX_LEN), dtype=torch.int64, device="cuda"),
           torch.empty((N_WALKS,), dtype=torch.int32, device="cuda"))
    sel = torch.from_numpy(ids).cuda()
    for form in FORMS:
        eng.set_scheduler(form)
        for bias, seed in ((_lib.BIAS_EXP, 12), (_lib.BIAS_UNIFORM, 13)):
            eng.walks(N_WALKS, MAX_LEN, bias=bias, seed=seed, out=out)
            runs[(form, bias)] = tuple(x.index_select(0, sel).cpu().numpy() for x in out)
    eng.close()
    del out, eng
    torch.cuda.empty_cache()
    orc = O.Oracle(spec.window, True)
    s = np.concatenate([h[0] for h in host])
    d = np.concatenate([h[1] for h in host])
    t = np.concatenate([h[2] for h in host])
    del host
    orc.ingest(s, d, t)
    del s, d, t
    ref = {b: orc.walks(ids=ids, max_len=MAX_LEN, bias=b, seed=sd, with_margin=(b == _lib.BIAS_EXP))
           for b, sd in ((_lib.BIAS_EXP, 12), (_lib.BIAS_UNIFORM, 13))}
    return runs, ref, orc.counts()


@pytest.mark.parametrize("form", FORMS)
def test_full_size_sampled_walks(full_size, form, record_property):
    runs, ref, counts = full_size
    assert counts["m"] >= 200_000_000
    g = runs[(form, _lib.BIAS_UNIFORM)]
    assert_walks_bit_exact(g, ref[_lib.BIAS_UNIFORM][:3], "uniform, form %d" % form)
    g = runs[(form, _lib.BIAS_EXP)]
    o = ref[_lib.BIAS_EXP]
    agree, total, div = compare_biased(g, o, o[3])
    # reported (pytest -rA / the junit record): how many sampled walks left
    # the oracle's path, and the margins (in double-evaluation bounds) where
    record_property("divergent_walks", len(div))
    record_property("divergent_margins", [round(m, 3) for _, _, m in div])
    print("form %d: %d of %d sampled exponential walks diverge (%d of %d hops agree), margins %s"
          % (form, len(div), SAMPLE, agree, total, [round(m, 3) for _, _, m in div]))
    assert total > SAMPLE  # the sample walks past its start edges
    assert agree / total >= MIN_HOP_AGREEMENT, (form, agree, total)
