"""Closed-form samplers (Sec. 2.5, Eq. 1-3) on the GPU vs the oracle.

The GPU evaluates uniform draws with integer arithmetic, exponential draws in
FP32 with an error bound and an FP64 fallback, and linear draws in FP64; all
must return the oracle's FP64 result.  Uniform and linear must agree on every
draw; exponential draws may differ only where the oracle's x is within twice
the double evaluation's own rounding bound of an integer (BOUND_UNITS).  The inputs mix random draws with draws
placed on and around the bucket boundaries, where a rounding slip would show.
"""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_16182_gb300 import _lib
from parity_util import BOUND_UNITS

pytestmark = pytest.mark.gpu
TWO53 = float(1 << 53)


def _random_inputs(rng, count):
    k = rng.integers(0, 1 << 53, count, dtype=np.int64).astype(np.uint64)
    kinds = rng.integers(0, 5, count)
    n = np.where(kinds == 0, rng.integers(1, 9, count),
        np.where(kinds == 1, rng.integers(1, 1000, count),
        np.where(kinds == 2, rng.integers(1, 1 << 20, count),
        np.where(kinds == 3, rng.integers(1, (1 << 31) - 1, count),
                 (1 << rng.integers(0, 31, count)) + rng.integers(-1, 2, count))))).astype(np.int64)
    n = np.clip(n, 1, (1 << 31) - 1)
    return k, n


def _uniform_boundaries(rng, count):
    """k with k*n within a few units of a multiple of 2^53 (the x = m edges)."""
    n = rng.integers(1, (1 << 31) - 1, count).astype(np.int64)
    n[: count // 4] = rng.integers(1, 64, count // 4)
    m = (rng.random(count) * n).astype(np.int64)
    k0 = np.array([-(-(int(mi) << 53) // int(ni)) for mi, ni in zip(m, n)], dtype=object)
    d = rng.integers(-3, 4, count)
    k = np.array([max(0, min((1 << 53) - 1, int(a) + int(b))) for a, b in zip(k0, d)], dtype=np.uint64)
    return k, n


def _linear_boundaries(rng, count):
    n = rng.integers(1, 1 << 20, count).astype(np.int64)
    i = (rng.random(count) * n).astype(np.int64)
    k = []
    for ii, nn in zip(i, n):
        num, den = int(ii) * (int(ii) + 1), int(nn) * (int(nn) + 1)
        k.append(min((1 << 53) - 1, max(0, (num << 53) // den + int(rng.integers(-3, 4)))))
    return np.array(k, dtype=np.uint64), n


def _exp_boundaries(rng, count, lam):
    n = rng.integers(1, 200, count).astype(np.int64)
    n[: count // 3] = rng.integers(1, 1 << 24, count // 3)
    i = np.minimum((rng.random(count) * 8).astype(np.int64), n - 1)
    i = n - 1 - i   # boundaries near the newest groups, where exp mass sits
    k = []
    for ii, nn in zip(i, n):
        # u at which the index steps from ii-1 to ii: (e^{lam ii} - 1) / (e^{lam n} - 1)
        a = lam * float(ii) - lam * float(nn)
        u = math.exp(a) * (1.0 - math.exp(-lam * ii)) / (1.0 - math.exp(-lam * nn)) if nn > 0 else 0.0
        kk = int(u * TWO53) + int(rng.integers(-2, 3))
        k.append(min((1 << 53) - 1, max(0, kk)))
    return np.array(k, dtype=np.uint64), n


def _gpu(eng, k, n, bias, lam):
    kd = torch.from_numpy(k.view(np.int64)).cuda()
    nd = torch.from_numpy(n).cuda()
    out = torch.empty(k.shape[0], dtype=torch.int64, device="cuda")
    _lib.tempest_sample_index(eng.h, kd.data_ptr(), nd.data_ptr(), k.shape[0], bias, lam, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def eng():
    e = _lib.Engine(window=0, device="cuda:0")
    yield e
    e.close()


@pytest.mark.parametrize("bias", [0, 1])
def test_uniform_and_linear_bit_exact(eng, bias):
    rng = np.random.default_rng(10 + bias)
    parts = [_random_inputs(rng, 2_000_000), _uniform_boundaries(rng, 200_000)]
    if bias == 1:
        parts.append(_linear_boundaries(rng, 200_000))
    k = np.concatenate([p[0] for p in parts])
    n = np.concatenate([p[1] for p in parts])
    got = _gpu(eng, k, n, bias, 1.0)
    want, _ = O.sampler_batch(k, n, bias)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, "first mismatch k=%d n=%d gpu=%d oracle=%d" % (k[bad[0]], n[bad[0]], got[bad[0]],
                                                                       want[bad[0]])
    assert ((got >= 0) & (got < n)).all()


@pytest.mark.parametrize("lam", [1.0, 0.5, 3.0, 1e-3, 1e-8])
def test_exponential_agrees_up_to_boundary(eng, lam):
    rng = np.random.default_rng(int(lam * 1000) + 7)
    parts = [_random_inputs(rng, 1_500_000), _exp_boundaries(rng, 150_000, lam)]
    k = np.concatenate([p[0] for p in parts])
    n = np.concatenate([p[1] for p in parts])
    got = _gpu(eng, k, n, 2, lam)
    want, margin = O.sampler_batch(k, n, 2, lam)
    bad = got != want
    assert (margin[bad] <= BOUND_UNITS).all(), "disagreement away from a boundary"
    assert bad.mean() <= 1e-4
    assert ((got >= 0) & (got < n)).all()


def _exp_band(n, lam, rng, mp):
    """Draws whose exact x lies 1e-12 ... 1e-4 (in x) on either side of a
    bucket edge: the band in which the GPU's FP32 bound alone decides (no
    FP64 fallback) once the distance exceeds that bound."""
    E = mp.exp(-lam * n)
    if lam >= 1.0:
        edges = [n - 1 - j for j in range(8)]
    elif lam * n > 20:
        edges = [n - int(rng.integers(1, int(20 / lam))) for _ in range(8)]
    else:
        edges = [int(rng.integers(1, n)) for _ in range(8)]
    ks = []
    for i in edges:
        if i <= 0:
            continue
        for d in (1e-12, 1e-11, 1e-10, 1e-9, 3e-9, 1e-8, 3e-8, 1e-7, 3e-7, 1e-6, 3e-6, 1e-5, 1e-4):
            for sgn in (-1, 1):
                x = mp.mpf(i) + sgn * mp.mpf(d)
                u = (mp.exp(lam * (x - n)) - E) / (1 - E)
                k = int(mp.nint(u * TWO53))
                if 0 < k < (1 << 53):
                    ks.append(k)
    return ks


@pytest.mark.parametrize("n", [10**6, 1 << 24, 10**8, (1 << 31) - 1])
def test_exponential_fp32_band(eng, n):
    """Exponential draws placed 1e-12 ... 1e-4 from a bucket edge, for n up
    to 2^31 - 1 and rates 1, 1e-3 and 1/n: the GPU decides most of them in
    FP32 with its error bound and must return the oracle's index on every
    draw more than BOUND_UNITS double-evaluation bounds from the edge."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    rng = np.random.default_rng(n % 1000 + 5)
    checked = 0
    for lam in (1.0, 1e-3, 1.0 / n):
        k = np.array(_exp_band(n, lam, rng, mp), dtype=np.uint64)
        nn = np.full(k.shape[0], n, np.int64)
        got = _gpu(eng, k, nn, 2, lam)
        want, margin = O.sampler_batch(k, nn, 2, lam)
        bad = got != want
        assert (margin[bad] <= BOUND_UNITS).all(), (
            "lambda %g: %d draws disagree beyond the bound (worst margin %g bounds)"
            % (lam, int((margin[bad] > BOUND_UNITS).sum()), float(margin[bad].max())))
        checked += int((margin > BOUND_UNITS).sum())
    # draws that must agree: most of the band lies beyond the double's bound
    assert checked > 80
