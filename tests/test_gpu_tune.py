"""Tuning knobs and the autotuner.

Every knob only remaps work to threads, so walks under any setting must be
bit-identical to walks under the defaults; the autotuner must report the
trials it timed and leave its choice selected.
"""
import pytest
import torch

from paper_2605_16182_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


def _engine():
    spec = synth.config_mid(scale=0.02)
    eng = _lib.Engine(window=spec.window, directed=True, device="cuda:0")
    for _, s, d, t in spec.batches(last=8):
        eng.ingest(s.cuda(), d.cuda(), t.cuda())
    return eng


def _walks(eng, bias, seed=9):
    return [x.clone() for x in eng.walks(20000, 30, bias=bias, seed=seed)]


def test_knobs_validate_and_round_trip():
    eng = _engine()
    for knob, bad in ((_lib.TUNE_BKT_LOG, 6), (_lib.TUNE_COOP_W_WARP, 0), (_lib.TUNE_COOP_MEGA, 100),
                      (_lib.TUNE_STREAM_CTAS, -1), (_lib.TUNE_PAD_PASS, 2), (_lib.TUNE_HOST_LINK_PCT, 101),
                      (_lib.TUNE_HOST_THREADS, -1), (_lib.TUNE_HOST_THREADS, 257), (17, 0)):
        with pytest.raises(_lib.TempestError) as e:
            eng.set_tuning(knob, bad)
        assert e.value.code == _lib.TEMPEST_EINVAL
    for knob, val in ((_lib.TUNE_BKT_LOG, 4), (_lib.TUNE_COOP_W_WARP, 16), (_lib.TUNE_COOP_MEGA, 2048),
                      (_lib.TUNE_STREAM_CTAS, 2), (_lib.TUNE_PAD_PASS, 1), (_lib.TUNE_HOST_LINK_PCT, 30),
                      (_lib.TUNE_HOST_THREADS, 3), (_lib.TUNE_HOST_THREADS, 0)):
        eng.set_tuning(knob, val)
        assert eng.get_tuning(knob) == val


@pytest.mark.parametrize("sched", [_lib.SCHED_STREAM, _lib.SCHED_COOP, _lib.SCHED_FULL_WALK, _lib.SCHED_GRAPH,
                                   _lib.SCHED_LANE])
def test_every_knob_setting_gives_the_same_walks(sched):
    eng = _engine()
    ref = {b: _walks(eng, b) for b in (0, 2)}
    eng.set_scheduler(sched)
    for knob, val in ((_lib.TUNE_BKT_LOG, 0), (_lib.TUNE_BKT_LOG, 5), (_lib.TUNE_COOP_W_WARP, 1),
                      (_lib.TUNE_COOP_W_WARP, 64), (_lib.TUNE_COOP_MEGA, 256), (_lib.TUNE_STREAM_CTAS, 1),
                      (_lib.TUNE_STREAM_CTAS, 5), (_lib.TUNE_PAD_PASS, 1), (_lib.TUNE_PAD_PASS, 0)):
        eng.set_tuning(knob, val)
        for b in (0, 2):
            got = eng.walks(20000, 30, bias=b, seed=9)
            assert all(torch.equal(x, y) for x, y in zip(ref[b], got)), (sched, knob, val, b)


def test_autotune_reports_and_keeps_its_choice():
    eng = _engine()
    ref = _walks(eng, 2)
    rep = eng.autotune(50000, 30, bias=2, seed=1, forms=True)
    assert len(rep["trials"]) >= 8
    assert rep["best_ms"] <= rep["start_ms"] + 1e-9
    assert rep["best_ms"] == min(t["ms"] for t in rep["trials"])
    assert {t["sched"] for t in rep["trials"]} == {0, 1, 2, 3, 4}
    assert eng.get_tuning(_lib.TUNE_BKT_LOG) == rep["bkt_log"]
    assert eng.get_tuning(_lib.TUNE_STREAM_CTAS) == rep["stream_ctas"]
    got = eng.walks(20000, 30, bias=2, seed=9)
    assert all(torch.equal(x, y) for x, y in zip(ref, got))
    with pytest.raises(_lib.TempestError):
        eng.autotune(0, 30)


def test_autotune_on_a_mixed_request():
    eng = _engine()
    g = torch.Generator().manual_seed(3)
    n = 30000
    lens = torch.randint(2, 41, (n,), generator=g, dtype=torch.int32).cuda()
    bias = torch.randint(0, 3, (n,), generator=g, dtype=torch.int32).to(torch.uint8).cuda()
    ref = [x.clone() for x in eng.walks_mixed(lens, bias, seed=8, max_len_cap=40)]
    rep = eng.autotune_mixed(lens, bias, max_len_cap=40, seed=2)
    assert len(rep["trials"]) >= 8 and rep["best_ms"] == min(t["ms"] for t in rep["trials"])
    got = eng.walks_mixed(lens, bias, seed=8, max_len_cap=40)
    assert all(torch.equal(x, y) for x, y in zip(ref, got))
    with pytest.raises(_lib.TempestError):
        eng.autotune_mixed(lens.cpu(), bias.cpu(), max_len_cap=40)


def test_autotune_per_ingest_charges_the_index_rebuild():
    """With the per-ingest flag every timed call rebuilds the derived walk
    indexes (as the first call after an ingest does); the walks stay the same
    and the reported times include the rebuild."""
    eng = _engine()
    ref = _walks(eng, 2)
    plain = eng.autotune(50000, 30, bias=2, seed=1, forms=False)
    rep = eng.autotune(50000, 30, bias=2, seed=1, forms=False, per_ingest=True)
    assert rep["best_ms"] == min(t["ms"] for t in rep["trials"])
    assert rep["start_ms"] >= 0.8 * plain["best_ms"]
    got = eng.walks(20000, 30, bias=2, seed=9)
    assert all(torch.equal(x, y) for x, y in zip(ref, got))
