"""Host-side logic of bench.py (no GPU): the clock-sample summary, the
percentile rule and the recorded-traffic lookup that feeds the roofline's
`traffic` key."""
import datetime
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _sampler(bench, tmp_path, rows, t_ref):
    """A sampler whose 'nvidia-smi' already wrote rows (dt seconds from t_ref,
    gpu index, SM MHz, sw_power_cap flag, hw_slowdown flag)."""
    s = bench.ClockSampler(str(tmp_path / "clocks.csv"))
    with open(s.path, "w") as f:
        for dt, idx, sm, cap, slow in rows:
            ts = datetime.datetime.fromtimestamp(t_ref + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            f.write("%s, %d, %d, 2070, 900.0, 0x0, %s, Not Active, Not Active, %s\n"
                    % (ts, idx, sm, "Active" if slow else "Not Active", "Active" if cap else "Not Active"))
        f.write("garbage line\n")
    s.proc = _Done()
    s.f = open(os.devnull, "w")
    return s


def test_clock_summary_keeps_the_timed_window(tmp_path):
    bench = _bench()
    t0 = 1.0e9
    rows = [(-2.0, 0, 900, False, True),   # before the window: a slowdown that must not count
            (0.01, 0, 2070, False, False),
            (0.06, 0, 2050, True, False),
            (0.11, 1, 1000, False, False),  # another GPU
            (0.12, 0, 2060, False, False),
            (3.0, 0, 800, False, False)]    # after the window
    out = _sampler(bench, tmp_path, rows, t0).stop(0, t0, t0 + 0.15)
    assert out["samples"] == 3 and out["window"] == "timed steps"
    assert out["sm_mhz"] == 2060 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_falls_back_to_all_samples(tmp_path):
    bench = _bench()
    t0 = 1.0e9
    rows = [(-1.0, 0, 2070, False, False), (-0.5, 0, 2000, False, True)]
    out = _sampler(bench, tmp_path, rows, t0).stop(0, t0, t0 + 0.1)
    assert out["samples"] == 2 and out["window"] == "autotune and timed steps"
    assert out["reasons"] == ["hw_slowdown"]
    assert _sampler(bench, tmp_path, [], t0).stop(0, t0, t0 + 1) is None


def test_percentile_rule():
    bench = _bench()
    assert bench.percentile([], 50) is None
    xs = [5.0, 1.0, 3.0, 2.0, 4.0]
    assert bench.percentile(xs, 50) == 3.0
    assert bench.percentile(xs, 0) == 1.0 and bench.percentile(xs, 100) == 5.0
    assert bench.percentile(list(range(101)), 99) == 99


def test_recorded_traffic_is_keyed_to_the_kernel_source(tmp_path, monkeypatch):
    """The roofline's traffic comes from a committed capture only while the
    walker source it was taken on is unchanged, and only for that kernel."""
    bench = _bench()
    fake_root = tmp_path / "root"
    (fake_root / "profiles").mkdir(parents=True)
    (fake_root / "paper_2605_16182_gb300").symlink_to(os.path.join(ROOT, "paper_2605_16182_gb300"))
    rec = {"kernel": "k_walks_lane<OneReq, 4>", "dram_bytes_per_hop": 550.0,
           "kernel_source_hash": bench.kernel_source_hash()}
    path = fake_root / "profiles" / "walk_kernel_traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    assert bench.recorded_traffic(1000.0, "k_walks_lane") == pytest.approx(550000.0)
    assert bench.recorded_traffic(1000.0, "k_walks_stream") is None
    path.write_text(json.dumps(dict(rec, kernel_source_hash="0" * 16)))
    assert bench.recorded_traffic(1000.0, "k_walks_lane") is None
    path.unlink()
    assert bench.recorded_traffic(1000.0, "k_walks_lane") is None


@pytest.mark.parametrize("steps,warmup", [(20, 5), (7, 3), (1, 1), (12, 0)])
def test_batch_plan_runs_any_step_count(steps, warmup):
    """The bench's batch plan for any --steps / --warmup: every step ingests
    BATCHES_PER_STEP full batches, in stream order, past the stream's nominal
    100 batches when the run is longer; timestamps never decrease across the
    whole run, and a batch continued past the end is the same as the one the
    generator gives for that edge range from scratch."""
    import torch
    from paper_2605_16182_gb300 import synth
    bench = _bench()
    spec = synth.config_billion(scale=1e-4)
    spec.n_nodes = 5000  # a small id table; the plan does not depend on it
    plan = bench.batch_plan(steps, warmup)
    assert len(plan) == steps + warmup
    assert [p[1] for p in plan] == [False] * warmup + [True] * steps
    feeder = bench.StepFeeder(spec, "cpu")
    last_ts = None
    n_batches = 0
    for step, timed, b0, b1 in plan:
        got = feeder.take(b0, b1)
        assert len(got) == bench.BATCHES_PER_STEP == b1 - b0
        for s, d, t in got:
            assert s.shape[0] == d.shape[0] == t.shape[0] == spec.batch
            assert bool((t[1:] >= t[:-1]).all())
            if last_ts is not None:
                assert int(t[0]) >= last_ts
            last_ts = int(t[-1])
        n_batches = b1
    assert n_batches == (steps + warmup) * bench.BATCHES_PER_STEP
    # the first batch past the stream's end equals the generator's own edges there
    k = spec.n_batches
    if n_batches > k:
        ref = spec.edges(k * spec.batch, spec.batch, "cpu")
        feeder2 = bench.StepFeeder(spec, "cpu")
        feeder2.take(0, k)
        (s, d, t), = feeder2.take(k, k + 1)
        assert torch.equal(s, ref[0]) and torch.equal(d, ref[1]) and torch.equal(t, ref[2])


def test_stream_refuses_batches_past_its_end():
    from paper_2605_16182_gb300 import synth
    spec = synth.config_billion(scale=1e-4)
    spec.n_nodes = 5000
    with pytest.raises(ValueError):
        list(spec.batches(first=98, last=101))
    with pytest.raises(ValueError):
        spec.edges(10, -1)
    assert len(list(spec.batches(first=98, last=101, extend=True))) == 3


def test_feeder_takes_batches_in_order():
    from paper_2605_16182_gb300 import synth
    bench = _bench()
    spec = synth.config_billion(scale=1e-4)
    spec.n_nodes = 5000
    f = bench.StepFeeder(spec, "cpu")
    f.take(0, 2)
    with pytest.raises(ValueError):
        f.take(5, 6)
