"""Python wrapper of the CPU oracle (tempest_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the cpu_baseline / reference
legs of ``bench.py`` may import this module.  It never imports the CUDA
library and the CUDA library never imports it.

The oracle follows the paper's definitions (Sec. 2.1 neighbourhood, Sec. 2.3
dual index, Sec. 2.5 samplers, Sec. 2.6 sliding window); see the header of
``tempest_oracle.c`` for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tempest_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")

BIAS_UNIFORM, BIAS_LINEAR, BIAS_EXP, BIAS_EXP_WEIGHT, BIAS_NODE2VEC = 0, 1, 2, 3, 4
N2V_MAX_TRIALS = 4096
START_UNIFORM_EDGE, START_BIASED_TS, START_PER_NODE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        vp, i64, i32, u64, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_uint64, ctypes.c_double)
        L.orc_create.restype = vp
        L.orc_create.argtypes = [i64, ctypes.c_int]
        L.orc_destroy.argtypes = [vp]
        L.orc_set_bias_params.argtypes = [vp, dbl, dbl]
        L.orc_ingest.argtypes = [vp, vp, vp, vp, i64]
        L.orc_walks.argtypes = [vp, i64, vp, i32, vp, i32, vp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, u64,
                                vp, vp, vp, vp, vp]
        L.orc_counts.argtypes = [vp, vp]
        L.orc_set_weight_rate.argtypes = [vp, dbl]
        L.orc_set_node2vec.argtypes = [vp, dbl, dbl]
        L.orc_weight_pick.argtypes = [vp, vp, i64, dbl, dbl, vp]
        L.orc_weight_pick.restype = i64
        L.orc_active_nodes.argtypes = [vp, vp]
        L.orc_active_nodes.restype = i64
        L.orc_export_live.argtypes = [vp, vp, vp, vp]
        L.orc_export_ts_groups.argtypes = [vp, vp]
        L.orc_export_node_view.argtypes = [vp, vp, vp, vp, vp]
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_u53.restype = dbl
        L.orc_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.orc_sampler_x.restype = dbl
        L.orc_sampler_x.argtypes = [dbl, i64, ctypes.c_int, dbl]
        L.orc_sampler_index.restype = i64
        L.orc_sampler_x_bound.restype = dbl
        L.orc_sampler_x_bound.argtypes = [dbl, i64, ctypes.c_int, dbl]
        L.orc_sampler_index.argtypes = [dbl, i64, ctypes.c_int, dbl]
        L.orc_sampler_batch.argtypes = [vp, vp, i64, ctypes.c_int, dbl, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u53(hi, lo):
    return lib().orc_u53(int(hi), int(lo))


def sampler_x(u, n, bias, lam=1.0):
    return lib().orc_sampler_x(float(u), int(n), int(bias), float(lam))


def sampler_index(u, n, bias, lam=1.0):
    return lib().orc_sampler_index(float(u), int(n), int(bias), float(lam))


def sampler_x_bound(u, n, bias, lam=1.0):
    """Bound on the rounding error of sampler_x's double evaluation (units of x)."""
    return lib().orc_sampler_x_bound(float(u), int(n), int(bias), float(lam))


def sampler_batch(k, n, bias, lam=1.0):
    """(index int64[count], margin float64[count]) for u = k * 2^-53; the
    margin is the distance of x to the nearest integer in units of
    sampler_x_bound."""
    k = np.ascontiguousarray(k, dtype=np.uint64)
    n = np.ascontiguousarray(n, dtype=np.int64)
    out = np.zeros(k.shape[0], np.int64)
    mg = np.zeros(k.shape[0], np.float64)
    lib().orc_sampler_batch(_p(k), _p(n), int(k.shape[0]), int(bias), float(lam), _p(out), _p(mg))
    return out, mg


class Oracle:
    """Single-threaded CPU restatement of the streaming engine."""

    COUNT_KEYS = ("m", "G_tot", "n_nodes", "M", "Gn", "dropped_late", "evicted",
                  "has_cutoff", "cutoff", "seq_next")

    def __init__(self, window: int = 0, directed: bool = True):
        self._h = lib().orc_create(int(window), 1 if directed else 0)
        if not self._h:
            raise MemoryError("orc_create")
        self.directed = directed

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_bias_params(self, lambda_hop: float, lambda_start: float = 0.0):
        rc = lib().orc_set_bias_params(self._h, float(lambda_hop), float(lambda_start))
        if rc != 0:
            raise ValueError("orc_set_bias_params rc=%d" % rc)

    def ingest(self, src, dst, ts):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        ts = np.ascontiguousarray(ts, dtype=np.int64)
        assert src.shape == dst.shape == ts.shape
        rc = lib().orc_ingest(self._h, _p(src), _p(dst), _p(ts), int(src.shape[0]))
        if rc != 0:
            raise ValueError("orc_ingest rc=%d" % rc)

    def counts(self) -> dict:
        out = np.zeros(10, np.int64)
        lib().orc_counts(self._h, _p(out))
        return dict(zip(self.COUNT_KEYS, (int(x) for x in out)))

    def state(self) -> dict:
        c = self.counts()
        m, G, N, M, Gn = c["m"], c["G_tot"], c["n_nodes"], c["M"], c["Gn"]
        src = np.zeros(m, np.int32)
        dst = np.zeros(m, np.int32)
        ts = np.zeros(m, np.int64)
        lib().orc_export_live(self._h, _p(src), _p(dst), _p(ts))
        tgo = np.zeros(G + 1, np.int64)
        lib().orc_export_ts_groups(self._h, _p(tgo))
        node_off = np.zeros(N + 1, np.int64)
        node_order = np.zeros(max(M, 1), np.int64)
        ngo = np.zeros(Gn + 1, np.int64)
        gidx = np.zeros(N + 1, np.int64)
        lib().orc_export_node_view(self._h, _p(node_off), _p(node_order), _p(ngo), _p(gidx))
        return dict(counts=c, src=src, dst=dst, ts=ts, ts_group_off=tgo, node_off=node_off,
                    node_order=node_order[:M], node_group_off=ngo, node_gidx=gidx)

    def set_weight_rate(self, lambda_w):
        if lib().orc_set_weight_rate(self._h, float(lambda_w)) != 0:
            raise ValueError("bad weight rate")

    def set_node2vec(self, p, q):
        """Return (p) and in-out (q) parameters of Temporal Node2Vec walks (bias 4)."""
        if lib().orc_set_node2vec(self._h, float(p), float(q)) != 0:
            raise ValueError("Node2Vec p, q must lie in [1e-3, 1e3]")

    def active_nodes(self, direction=0):
        """Nodes with at least one live entry in the node view (the in-view for
        direction 1: a live in-edge), in id order."""
        if direction == 1:
            st = self.state()
            src, dst = np.asarray(st["src"]), np.asarray(st["dst"])
            nodes = dst if self.directed else np.concatenate([src, dst])
            return np.unique(nodes).astype(np.int32)
        n = int(lib().orc_active_nodes(self._h, None))
        out = np.zeros(max(n, 1), np.int32)
        lib().orc_active_nodes(self._h, _p(out))
        return out[:n]

    def walks(self, n_walks=None, max_len=2, bias=BIAS_UNIFORM, start_policy=START_UNIFORM_EDGE,
              seed=0, ids=None, max_len_arr=None, bias_arr=None, with_margin=False,
              with_bytes=False, walks_per_node=None, direction=0):
        """Returns (node [n, cap], ts [n, cap], len [n], margin or None, bytes or None).
        With START_PER_NODE, walk w starts at active node w // walks_per_node
        (by default n_walks divided by the number of active nodes)."""
        if ids is not None:
            ids = np.ascontiguousarray(ids, dtype=np.int64)
            n = ids.shape[0]
        else:
            n = int(n_walks)
        k = 0
        if start_policy == START_PER_NODE:
            if walks_per_node is None:
                na = len(self.active_nodes(direction))
                if na == 0 or n % na:
                    raise ValueError("per-node walks: %d walks for %d active nodes" % (n, na))
                walks_per_node = n // na
            k = int(walks_per_node)
        cap = int(max_len)
        if max_len_arr is not None:
            max_len_arr = np.ascontiguousarray(max_len_arr, dtype=np.int32)
            cap = max(cap, int(max_len_arr.max()) if n else 2)
        if bias_arr is not None:
            bias_arr = np.ascontiguousarray(bias_arr, dtype=np.uint8)
        node = np.zeros((n, cap), np.int32)
        ts = np.zeros((n, cap), np.int64)
        ln = np.zeros(n, np.int32)
        margin = np.zeros((n, cap), np.float64) if with_margin else None
        nbytes = np.zeros(1, np.float64) if with_bytes else None
        rc = lib().orc_walks(self._h, n, _p(ids), cap, _p(max_len_arr), int(max_len), _p(bias_arr),
                             int(bias), int(start_policy), k, int(direction), ctypes.c_uint64(int(seed) & (2**64 - 1)),
                             _p(node), _p(ts), _p(ln), _p(margin), _p(nbytes))
        if rc != 0:
            raise ValueError("orc_walks rc=%d" % rc)
        return node, ts, ln, margin, (float(nbytes[0]) if with_bytes else None)


def weight_pick(ts, size, lam, u):
    """The weight-based sampler over groups with timestamps ts and sizes size
    (ascending): (group index, relative margin of the draw)."""
    ts = np.ascontiguousarray(ts, dtype=np.int64)
    size = np.ascontiguousarray(size, dtype=np.int64)
    mg = np.zeros(1, np.float64)
    j = int(lib().orc_weight_pick(_p(ts), _p(size), int(ts.shape[0]), float(lam), float(u), _p(mg)))
    return j, float(mg[0])
