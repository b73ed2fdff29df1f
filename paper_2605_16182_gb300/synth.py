"""Seeded synthetic edge streams shared by the tests and the benchmark.

This module produces inputs only; it holds none of the engine's arithmetic
(no windowing, indexing, search or sampling of walks).  Every draw is a
counter-based hash of (seed, stream, index) evaluated with int64 tensor ops,
so the same call gives bit-identical arrays on the CPU and on a GPU.

Workload shapes (stand-ins for the paper's Alibaba / TGB / Konect streams,
none of which are reproduced):
  * node ids: Zipf(alpha) over ranks 1..N, sampled by integer search in a
    cumulative threshold table, then mapped through an affine bijection of
    [0, N) so that the hubs are not at id 0.  Sources and destinations are
    drawn independently through the same bijection, so the busiest sender is
    also the busiest receiver.
  * timestamps: either iid uniform integers, or a Poisson-like arrival
    process: exponential inter-arrival gaps (integer ns) from a 65536-bucket
    piecewise-linear inverse CDF of Exp(1) (truncated at ln 2^24 ~ 16.6
    means), scaled by a per-segment mean gap, then prefix-summed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Iterator, List, Optional

import numpy as np
import torch

_M64 = (1 << 64) - 1


def _s64(x: int) -> int:
    """Python int -> the int64 with the same 64-bit pattern."""
    x &= _M64
    return x - (1 << 64) if x >= (1 << 63) else x


_GOLD = _s64(0x9E3779B97F4A7C15)
_C1 = _s64(0xBF58476D1CE4E5B9)
_C2 = _s64(0x94D049BB133111EB)


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def mix64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on int64 tensors."""
    z = z + _GOLD
    z = (z ^ _srl(z, 30)) * _C1
    z = (z ^ _srl(z, 27)) * _C2
    return z ^ _srl(z, 31)


def u64(seed: int, stream: int, start: int, n: int, device) -> torch.Tensor:
    """n pseudo-random 64-bit words (as int64) for indices start..start+n-1."""
    base = mix64(torch.tensor([_s64(seed * 0x100000001B3 + stream * 0x9E37 + 12345)],
                              dtype=torch.int64, device=device))
    idx = torch.arange(start, start + n, dtype=torch.int64, device=device)
    return mix64(idx * _GOLD + base)


def u63(seed, stream, start, n, device) -> torch.Tensor:
    return _srl(u64(seed, stream, start, n, device), 1)


# --------------------------------------------------------------------------
# Zipf node ids
# --------------------------------------------------------------------------
_ZIPF_CACHE = {}


def zipf_thresholds(N: int, alpha: float) -> torch.Tensor:
    """int64 table thr[k] = floor(2^63 * P(rank <= k+1)), thr[N-1] = 2^63-1."""
    key = (int(N), float(alpha))
    t = _ZIPF_CACHE.get(key)
    if t is None:
        w = np.arange(1, N + 1, dtype=np.float64)
        np.power(w, -alpha, out=w)
        np.cumsum(w, out=w)
        w /= w[-1]
        thr = np.minimum(w * 9.223372036854775807e18, 9.2233720368547748e18).astype(np.int64)
        thr[-1] = (1 << 63) - 1
        t = torch.from_numpy(thr)
        _ZIPF_CACHE.clear()
        _ZIPF_CACHE[key] = t
    return t


def _coprime_multiplier(N: int) -> int:
    for a in (2654435761, 2246822519, 3266489917, 668265263, 374761393, 1103515245):
        if math.gcd(a % N if N > 1 else 1, N) == 1 and a % N != 0:
            return a % N
    a = N // 2 + 1
    while math.gcd(a, N) != 1:
        a += 1
    return a


_ZIPF_DEVICE = {}


def _thresholds_on(N: int, alpha: float, device) -> torch.Tensor:
    """zipf_thresholds on `device`, kept there for the next call (the table of
    a 100M-node stream is 800 MB)."""
    dev = torch.device(device)
    key = (int(N), float(alpha), str(dev))
    t = _ZIPF_DEVICE.get(key)
    if t is None:
        t = zipf_thresholds(N, alpha).to(dev)
        _ZIPF_DEVICE.clear()
        _ZIPF_DEVICE[key] = t
    return t


def zipf_ids(N: int, alpha: float, seed: int, stream: int, start: int, n: int, device,
             perm_seed: Optional[int] = None) -> torch.Tensor:
    """n Zipf(alpha) node ids in [0, N) as int32."""
    thr = _thresholds_on(N, alpha, device)
    u = u63(seed, stream, start, n, device)
    rank = torch.searchsorted(thr, u, right=True).clamp_(max=N - 1)
    ps = seed if perm_seed is None else perm_seed
    a = _coprime_multiplier(N)
    b = int(mix64(torch.tensor([_s64(ps)], dtype=torch.int64)).item()) % N
    ids = (rank * a + b) % N
    return ids.to(torch.int32)


# --------------------------------------------------------------------------
# timestamps
# --------------------------------------------------------------------------
_EXP_TABLE = None
_EXP_FRAC = 32  # fixed-point fraction bits of the Exp(1) table


def _exp_table() -> torch.Tensor:
    """Exp(1) quantiles -ln(1 - k/65536) in 32.32 fixed point, k = 0..65536
    (the last entry truncates the tail at ln 2^24)."""
    global _EXP_TABLE
    if _EXP_TABLE is None:
        k = np.arange(65537, dtype=np.float64)
        q = np.empty_like(k)
        q[:-1] = -np.log1p(-k[:-1] / 65536.0)
        q[-1] = 24.0 * math.log(2.0)
        _EXP_TABLE = torch.from_numpy(np.floor(q * 2.0 ** _EXP_FRAC).astype(np.int64))
    return _EXP_TABLE


def exp_gaps(mean_gap: torch.Tensor, seed: int, stream: int, start: int, n: int, device) -> torch.Tensor:
    """Integer inter-arrival gaps ~ floor(mean * Exp(1)); mean_gap int64 per edge."""
    tab = _exp_table().to(device)
    u = u63(seed, stream, start, n, device)
    k = _srl(u, 47)                       # top 16 bits
    frac = (u >> 27) & ((1 << 20) - 1)    # next 20 bits
    lo = tab[k]
    hi = tab[k + 1]
    e = lo + (((hi - lo) * frac) >> 20)   # Exp(1) in 32.32 fixed point
    return (e * mean_gap) >> _EXP_FRAC


def uniform_ts(R: int, seed: int, stream: int, start: int, n: int, device) -> torch.Tensor:
    return u63(seed, stream, start, n, device) % R


# --------------------------------------------------------------------------
# workload configurations
# --------------------------------------------------------------------------
@dataclass
class StreamSpec:
    """A synthetic edge stream split into equal batches."""
    name: str
    n_nodes: int
    n_edges: int
    alpha: float
    seed: int
    batch: int
    ts_kind: str = "poisson"           # "poisson" | "uniform"
    ts_range: int = 1_000_000          # uniform timestamps in [0, ts_range)
    mean_gaps: List[int] = field(default_factory=lambda: [1000])
    switch_every: int = 0              # alternate mean gap every this many edges
    t0: int = 1_000_000_000
    window: int = 0                    # engine window (< 0: count of newest edges kept)

    @property
    def n_batches(self) -> int:
        return (self.n_edges + self.batch - 1) // self.batch

    def mean_gap(self, start: int, n: int, device) -> torch.Tensor:
        if len(self.mean_gaps) == 1 or self.switch_every <= 0:
            return torch.full((n,), int(self.mean_gaps[0]), dtype=torch.int64, device=device)
        idx = torch.arange(start, start + n, dtype=torch.int64, device=device)
        seg = (idx // self.switch_every) % len(self.mean_gaps)
        return torch.tensor(self.mean_gaps, dtype=torch.int64, device=device)[seg]

    def edges(self, start: int, n: int, device="cpu", ts_base: Optional[int] = None):
        """Edges start..start+n-1 as (src int32, dst int32, ts int64).

        For Poisson streams the timestamps are a prefix sum of all gaps from
        edge 0, so ts_base (the timestamp of edge start-1, or t0 when
        start == 0) may be passed to avoid recomputing the prefix."""
        if start < 0 or n < 0:
            raise ValueError("edge range start %d, count %d" % (start, n))
        src = zipf_ids(self.n_nodes, self.alpha, self.seed, 1, start, n, device)
        dst = zipf_ids(self.n_nodes, self.alpha, self.seed, 2, start, n, device,
                       perm_seed=self.seed)
        if self.ts_kind == "uniform":
            ts = uniform_ts(self.ts_range, self.seed, 3, start, n, device)
        else:
            if ts_base is None:
                ts_base = self.ts_before(start, device)
            g = exp_gaps(self.mean_gap(start, n, device), self.seed, 3, start, n, device)
            ts = torch.cumsum(g, 0) + ts_base
        return src, dst, ts

    def ts_before(self, start: int, device="cpu", chunk: int = 1 << 24) -> int:
        """Timestamp of edge start-1 (t0 for start == 0)."""
        t = self.t0
        s = 0
        while s < start:
            n = min(chunk, start - s)
            g = exp_gaps(self.mean_gap(s, n, device), self.seed, 3, s, n, device)
            t += int(g.sum().item())
            s += n
        return t

    def batches(self, device="cpu", first: int = 0, last: Optional[int] = None,
                extend: bool = False, ts_base: Optional[int] = None) -> Iterator:
        """Yield (k, src, dst, ts) for batches first..last-1.

        The stream holds n_batches batches (the last one possibly short).  A
        batch past the end raises ValueError unless extend is set: then the
        same generator continues past n_edges and every batch is full (the
        counter of every draw is the edge index, so a full batch k is the same
        whichever call produces it).  ts_base, for Poisson streams, is the
        timestamp of the edge before batch `first` (saves recomputing the
        prefix of gaps)."""
        last = self.n_batches if last is None else last
        if first < 0 or last < first:
            raise ValueError("batch range [%d, %d) is empty or negative" % (first, last))
        if last > self.n_batches and not extend:
            raise ValueError("the stream %s has %d batches; batches up to %d were asked for (extend=True "
                             "continues it)" % (self.name, self.n_batches, last))
        start = first * self.batch
        if self.ts_kind != "uniform" and ts_base is None:
            ts_base = self.ts_before(start, device)
        for k in range(first, last):
            s = k * self.batch
            n = self.batch if extend else min(self.batch, self.n_edges - s)
            src, dst, ts = self.edges(s, n, device, ts_base)
            if self.ts_kind != "uniform":
                ts_base = int(ts[-1].item()) if n else ts_base
            yield k, src, dst, ts


def walk_max_lens(n: int, lo: int, hi: int, seed: int, device="cpu") -> torch.Tensor:
    """Per-walk max_len uniform in [lo, hi] (int32)."""
    return (lo + u63(seed, 7, 0, n, device) % (hi - lo + 1)).to(torch.int32)


# the workloads the engine is measured on (sizes as stated by the benchmark spec)
def config_small(scale: float = 1.0) -> StreamSpec:
    """Directed, 10k nodes, 100k edges, Zipf 2.0, ts iid uniform in [0, 1e6), one batch."""
    e = max(1, int(100_000 * scale))
    return StreamSpec("plain-small-10k-nodes-100k-edges", 10_000, e, 2.0, 1001, e,
                      ts_kind="uniform", ts_range=1_000_000, window=0)


def config_mid(scale: float = 1.0) -> StreamSpec:
    """1M nodes, 20M edges, Zipf 2.1, Poisson gaps mean 1000 ns, 20 batches of 1M."""
    b = max(1, int(1_000_000 * scale))
    return StreamSpec("biased-mid-1M-nodes-20M-edges", 1_000_000, 20 * b, 2.1, 1002, b,
                      mean_gaps=[1000], window=-5 * b)


def config_billion(scale: float = 1.0) -> StreamSpec:
    """100M nodes, 1B edges, Zipf 2.0, bursty gaps (mean 1000/100 ns switching
    every 1e7 edges), 100 batches of 10M."""
    b = max(1, int(10_000_000 * scale))
    return StreamSpec("billion-edge-stream-100M-nodes-1B-edges", 100_000_000, 100 * b, 2.0, 1003, b,
                      mean_gaps=[1000, 100], switch_every=b, window=-20 * b)


def config_undirected_batched(scale: float = 1.0) -> StreamSpec:
    """Undirected, 10M nodes, 200M edges, Zipf 1.9, Poisson mean 1000 ns, one batch."""
    e = max(1, int(200_000_000 * scale))
    return StreamSpec("batched-undirected-10M-nodes-200M-edges", 10_000_000, e, 1.9, 1004, e,
                      mean_gaps=[1000], window=0)
