"""ctypes binding of libtempest.so (include/tempest.h).

Argument marshalling only: every step of ingest and walk generation runs in
the CUDA library.  If the library is missing this module raises; there is no
CPU fallback.  The module-level functions carry the C names; ``Engine`` wraps
a handle for torch tensors / numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

TEMPEST_OK = 0
TEMPEST_EINVAL = -1
TEMPEST_ENOMEM = -2
TEMPEST_ECUDA = -3
TEMPEST_ETIMEDOUT = -4
TEMPEST_EBUSY = -5

BIAS_UNIFORM, BIAS_LINEAR, BIAS_EXP, BIAS_EXP_WEIGHT, BIAS_NODE2VEC = 0, 1, 2, 3, 4
N2V_MAX_TRIALS = 4096
START_UNIFORM_EDGE, START_BIASED_TS, START_PER_NODE = 0, 1, 2
SCHED_FULL_WALK, SCHED_COOP, SCHED_STREAM, SCHED_GRAPH, SCHED_LANE = 0, 1, 2, 3, 4
(TUNE_BKT_LOG, TUNE_COOP_W_WARP, TUNE_COOP_MEGA, TUNE_STREAM_CTAS, TUNE_PAD_PASS, TUNE_HOST_LINK_PCT,
 TUNE_HOST_THREADS, TUNE_EVICT, TUNE_MIRROR_MIN) = 0, 1, 2, 3, 4, 5, 6, 7, 8
TUNE_FORMS = 1
TUNE_PER_INGEST = 2
TUNE_MAX_TRIALS = 48
(STATE_SRC, STATE_DST, STATE_TS, STATE_TS_GROUP_OFF, STATE_NODE_OFF, STATE_NODE_ORDER,
 STATE_NODE_GROUP_OFF, STATE_NODE_GIDX) = range(8)

# every function declared in include/tempest.h
EXPORTED = (
    "tempest_create", "tempest_destroy", "tempest_set_stream", "tempest_set_allocator",
    "tempest_set_bias_params", "tempest_ingest", "tempest_walks", "tempest_walks_mixed",
    "tempest_set_scheduler", "tempest_last_walk_stats", "tempest_get_counts",
    "tempest_export_state", "tempest_sync", "tempest_last_error", "tempest_version",
    "tempest_sort_batch_noalloc", "tempest_sample_index", "tempest_walks_batch",
    "tempest_server_create", "tempest_server_destroy", "tempest_server_submit_walks",
    "tempest_server_submit_ingest", "tempest_server_progress", "tempest_server_status",
    "tempest_server_release", "tempest_server_drain", "tempest_server_stats",
    "tempest_set_tuning", "tempest_get_tuning", "tempest_autotune", "tempest_autotune_mixed",
    "tempest_active_nodes", "tempest_set_weight_rate", "tempest_enable_backward", "tempest_walks_backward",
    "tempest_active_nodes_backward", "tempest_set_node2vec",
)
NOALLOC_MAX_EDGES = 262144


class TempestError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("tempest error %d: %s" % (code, msg))
        self.code = code


class IngestStats(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int64), ("n_dropped_late", ctypes.c_int64),
                ("n_evicted", ctypes.c_int64), ("n_live", ctypes.c_int64),
                ("n_ts_groups", ctypes.c_int64), ("n_node_groups", ctypes.c_int64),
                ("n_nodes", ctypes.c_int64), ("cutoff", ctypes.c_int64),
                ("has_cutoff", ctypes.c_int32), ("sorted_input", ctypes.c_int32),
                ("launches", ctypes.c_int64), ("evict_ms", ctypes.c_double),
                ("model_bytes", ctypes.c_int64), ("view_rebuilt", ctypes.c_int32), ("copied_ahead", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class WalkStats(ctypes.Structure):
    _fields_ = [("n_walks", ctypes.c_int64), ("hops", ctypes.c_int64),
                ("model_bytes", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("tier_launches", ctypes.c_int64 * 5), ("kernel_ms", ctypes.c_double),
                ("d2h_bytes", ctypes.c_int64), ("host_ms", ctypes.c_double * 3)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["tier_launches"] = list(self.tier_launches)
        d["host_ms"] = list(self.host_ms)
        return d


class TuneTrial(ctypes.Structure):
    _fields_ = [("sched", ctypes.c_int32), ("bkt_log", ctypes.c_int32), ("coop_w_warp", ctypes.c_int32),
                ("coop_mega", ctypes.c_int32), ("stream_ctas", ctypes.c_int32), ("pad_pass", ctypes.c_int32),
                ("ms", ctypes.c_double)]


class TuneReport(ctypes.Structure):
    _fields_ = [("sched", ctypes.c_int32), ("bkt_log", ctypes.c_int32), ("coop_w_warp", ctypes.c_int32),
                ("coop_mega", ctypes.c_int32), ("stream_ctas", ctypes.c_int32), ("pad_pass", ctypes.c_int32),
                ("n_trials", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("start_ms", ctypes.c_double),
                ("trials", TuneTrial * TUNE_MAX_TRIALS)]

    def as_dict(self):
        keys = ("sched", "bkt_log", "coop_w_warp", "coop_mega", "stream_ctas", "pad_pass")
        d = {k: getattr(self, k) for k in keys + ("best_ms", "start_ms")}
        d["trials"] = [dict({k: getattr(t, k) for k in keys}, ms=t.ms) for t in self.trials[:self.n_trials]]
        return d


class WalkRequest(ctypes.Structure):
    _fields_ = [("n_walks", ctypes.c_int64), ("max_len", ctypes.c_int32), ("bias", ctypes.c_int32),
                ("max_len_arr", ctypes.c_void_p), ("bias_arr", ctypes.c_void_p),
                ("start_policy", ctypes.c_int32), ("direction", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("node", ctypes.c_void_p), ("ts", ctypes.c_void_p), ("len", ctypes.c_void_p)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_L = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libtempest.so; raises if it has not been built."""
    global _L
    if _L is not None:
        return _L
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libtempest.so is not built (%s); run paper_2605_16182_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    vp, i64, i32, u64, dbl, ci = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_int)
    L.tempest_create.argtypes = [i64, ci, ctypes.POINTER(vp)]
    L.tempest_destroy.argtypes = [vp]
    L.tempest_set_stream.argtypes = [vp, vp]
    L.tempest_set_allocator.argtypes = [vp, ALLOC_FN, RELEASE_FN, vp, ctypes.c_size_t]
    L.tempest_set_bias_params.argtypes = [vp, dbl, dbl]
    L.tempest_ingest.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(IngestStats)]
    L.tempest_walks.argtypes = [vp, i64, i32, ci, ci, u64, vp, vp, vp]
    L.tempest_walks_mixed.argtypes = [vp, i64, vp, i32, vp, ci, u64, vp, vp, vp]
    L.tempest_set_scheduler.argtypes = [vp, ci]
    L.tempest_set_tuning.argtypes = [vp, ci, i64]
    L.tempest_get_tuning.argtypes = [vp, ci, ctypes.POINTER(i64)]
    L.tempest_autotune.argtypes = [vp, i64, ctypes.c_int32, ci, ci, ctypes.c_uint64, ctypes.c_int32,
                                   ctypes.POINTER(TuneReport)]
    L.tempest_active_nodes.argtypes = [vp, ctypes.POINTER(i64)]
    L.tempest_set_weight_rate.argtypes = [vp, dbl]
    L.tempest_enable_backward.argtypes = [vp]
    L.tempest_set_node2vec.argtypes = [vp, dbl, dbl]
    L.tempest_walks_backward.argtypes = [vp, i64, i32, ci, ci, u64, vp, vp, vp]
    L.tempest_active_nodes_backward.argtypes = [vp, ctypes.POINTER(i64)]
    L.tempest_autotune_mixed.argtypes = [vp, i64, vp, ctypes.c_int32, vp, ci, ctypes.c_uint64, ctypes.c_int32,
                                         ctypes.POINTER(TuneReport)]
    L.tempest_last_walk_stats.argtypes = [vp, ctypes.POINTER(WalkStats)]
    L.tempest_get_counts.argtypes = [vp, vp]
    L.tempest_export_state.argtypes = [vp, ci, vp, i64, ctypes.POINTER(i64)]
    L.tempest_sync.argtypes = [vp]
    L.tempest_last_error.argtypes = [vp]
    L.tempest_last_error.restype = ctypes.c_char_p
    L.tempest_version.restype = ctypes.c_char_p
    L.tempest_sort_batch_noalloc.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
    L.tempest_sample_index.argtypes = [vp, vp, vp, i64, ci, dbl, vp]
    L.tempest_walks_batch.argtypes = [vp, ctypes.POINTER(WalkRequest), ci]
    L.tempest_server_create.argtypes = [vp, ctypes.c_size_t, i64, ci, ctypes.POINTER(vp)]
    L.tempest_server_destroy.argtypes = [vp]
    L.tempest_server_submit_walks.argtypes = [vp, ctypes.POINTER(WalkRequest), ctypes.POINTER(ctypes.c_uint64)]
    L.tempest_server_submit_ingest.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(ctypes.c_uint64)]
    L.tempest_server_progress.argtypes = [vp, ctypes.POINTER(ci)]
    L.tempest_server_status.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ci), ctypes.POINTER(vp),
                                        ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(dbl)]
    L.tempest_server_release.argtypes = [vp, ctypes.c_uint64]
    L.tempest_server_drain.argtypes = [vp]
    L.tempest_server_stats.argtypes = [vp, vp]
    for name in EXPORTED:
        if name not in ("tempest_last_error", "tempest_version"):
            getattr(L, name).restype = ci
    _L = L
    return L


def _check(h, rc):
    if rc != TEMPEST_OK:
        msg = load().tempest_last_error(h)
        raise TempestError(rc, msg.decode() if msg else "")
    return rc


# ---------------------------------------------------------------- C names
def tempest_version() -> str:
    return load().tempest_version().decode()


def tempest_create(window: int, directed: bool):
    h = ctypes.c_void_p()
    _check(None, load().tempest_create(int(window), 1 if directed else 0, ctypes.byref(h)))
    return h


def tempest_destroy(h):
    return load().tempest_destroy(h)


def tempest_set_stream(h, stream_ptr: int):
    return _check(h, load().tempest_set_stream(h, ctypes.c_void_p(stream_ptr)))


def tempest_set_allocator(h, alloc, release, ctx, budget: int):
    return _check(h, load().tempest_set_allocator(h, alloc, release, ctx, ctypes.c_size_t(budget)))


def tempest_set_bias_params(h, lambda_hop: float, lambda_start: float):
    return _check(h, load().tempest_set_bias_params(h, float(lambda_hop), float(lambda_start)))


def tempest_ingest(h, src_ptr, dst_ptr, ts_ptr, n: int) -> IngestStats:
    st = IngestStats()
    _check(h, load().tempest_ingest(h, ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr),
                                    ctypes.c_void_p(ts_ptr), int(n), ctypes.byref(st)))
    return st


def tempest_walks(h, n_walks, max_len, bias, start_policy, seed, node_ptr, ts_ptr, len_ptr):
    return _check(h, load().tempest_walks(h, int(n_walks), int(max_len), int(bias), int(start_policy),
                                          ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                          ctypes.c_void_p(node_ptr), ctypes.c_void_p(ts_ptr),
                                          ctypes.c_void_p(len_ptr)))


def tempest_walks_backward(h, n_walks, max_len, bias, start_policy, seed, node_ptr, ts_ptr, len_ptr):
    return _check(h, load().tempest_walks_backward(h, int(n_walks), int(max_len), int(bias), int(start_policy),
                                                   ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                                   ctypes.c_void_p(node_ptr), ctypes.c_void_p(ts_ptr),
                                                   ctypes.c_void_p(len_ptr)))


def tempest_walks_mixed(h, n_walks, max_len_ptr, max_len_cap, bias_ptr, start_policy, seed, node_ptr,
                        ts_ptr, len_ptr):
    return _check(h, load().tempest_walks_mixed(h, int(n_walks), ctypes.c_void_p(max_len_ptr),
                                                int(max_len_cap), ctypes.c_void_p(bias_ptr),
                                                int(start_policy),
                                                ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                                ctypes.c_void_p(node_ptr), ctypes.c_void_p(ts_ptr),
                                                ctypes.c_void_p(len_ptr)))


def tempest_sample_index(h, u_bits_ptr, n_ptr, count, bias, lam, out_ptr):
    return _check(h, load().tempest_sample_index(h, ctypes.c_void_p(u_bits_ptr), ctypes.c_void_p(n_ptr),
                                                 int(count), int(bias), float(lam), ctypes.c_void_p(out_ptr)))


def make_request(n_walks, max_len, bias=0, start_policy=0, seed=0, node=None, ts=None, ln=None,
                 max_len_arr=None, bias_arr=None, direction=0) -> WalkRequest:
    """A tempest_walk_request; outputs / per-walk arrays are CUDA tensors or None."""
    r = WalkRequest()
    r.direction = int(direction)
    r.n_walks, r.max_len, r.bias, r.start_policy = int(n_walks), int(max_len), int(bias), int(start_policy)
    r.seed = int(seed) & (2**64 - 1)
    r.max_len_arr = _ptr(max_len_arr, "int32")
    r.bias_arr = _ptr(bias_arr, "uint8")
    r.node, r.ts, r.len = _ptr(node, "int32"), _ptr(ts, "int64"), _ptr(ln, "int32")
    return r


def tempest_walks_batch(h, reqs):
    arr = (WalkRequest * len(reqs))(*reqs)
    return _check(h, load().tempest_walks_batch(h, arr, len(reqs)))


class Server:
    """The serving loop of include/tempest.h (tempest_server_*)."""

    QUEUED, RUNNING, DONE = 0, 1, 2

    def __init__(self, engine, arena_bytes: int, max_wave_walks: int, max_inflight: int = 2):
        self.engine = engine
        self.s = ctypes.c_void_p()
        _check(engine.h, load().tempest_server_create(engine.h, ctypes.c_size_t(int(arena_bytes)),
                                                      int(max_wave_walks), int(max_inflight),
                                                      ctypes.byref(self.s)))

    def close(self):
        if self.s:
            load().tempest_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit_walks(self, req: WalkRequest) -> int:
        t = ctypes.c_uint64()
        _check(self.engine.h, load().tempest_server_submit_walks(self.s, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def submit_ingest(self, src, dst, ts) -> int:
        t = ctypes.c_uint64()
        _check(self.engine.h, load().tempest_server_submit_ingest(
            self.s, _ptr(src, "int32"), _ptr(dst, "int32"), _ptr(ts, "int64"), int(src.shape[0]),
            ctypes.byref(t)))
        return t.value

    def progress(self) -> int:
        n = ctypes.c_int()
        _check(self.engine.h, load().tempest_server_progress(self.s, ctypes.byref(n)))
        return n.value

    def status(self, ticket: int):
        st, lat = ctypes.c_int(), ctypes.c_double()
        node, ts, ln = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(self.engine.h, load().tempest_server_status(self.s, ctypes.c_uint64(ticket), ctypes.byref(st),
                                                           ctypes.byref(node), ctypes.byref(ts),
                                                           ctypes.byref(ln), ctypes.byref(lat)))
        return st.value, (node.value, ts.value, ln.value), lat.value

    def result(self, ticket: int, n_walks: int, max_len: int):
        """Copies of a finished walk request's outputs as torch tensors."""
        import torch
        st, (pn, pt, pl), _ = self.status(ticket)
        assert st == self.DONE, st

        class _View:
            def __init__(self, ptr, shape, typestr):
                self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                                 "version": 3, "strides": None}

        node = torch.as_tensor(_View(pn, (n_walks, max_len), "<i4"), device="cuda").clone()
        ts = torch.as_tensor(_View(pt, (n_walks, max_len), "<i8"), device="cuda").clone()
        ln = torch.as_tensor(_View(pl, (n_walks,), "<i4"), device="cuda").clone()
        return node, ts, ln

    def release(self, ticket: int):
        _check(self.engine.h, load().tempest_server_release(self.s, ctypes.c_uint64(ticket)))

    def drain(self):
        _check(self.engine.h, load().tempest_server_drain(self.s))

    def stats(self) -> dict:
        out = (ctypes.c_int64 * 4)()
        _check(self.engine.h, load().tempest_server_stats(self.s, out))
        return dict(waves=out[0], wave_requests=out[1], ingests=out[2], queued=out[3])


def tempest_set_scheduler(h, mode: int):
    return _check(h, load().tempest_set_scheduler(h, int(mode)))


def tempest_set_tuning(h, knob: int, value: int):
    return _check(h, load().tempest_set_tuning(h, int(knob), int(value)))


def tempest_get_tuning(h, knob: int) -> int:
    v = ctypes.c_int64()
    _check(h, load().tempest_get_tuning(h, int(knob), ctypes.byref(v)))
    return v.value


def tempest_active_nodes(h, direction=0) -> int:
    n = ctypes.c_int64()
    fn = load().tempest_active_nodes_backward if direction else load().tempest_active_nodes
    _check(h, fn(h, ctypes.byref(n)))
    return n.value


def tempest_enable_backward(h):
    return _check(h, load().tempest_enable_backward(h))


def tempest_autotune_mixed(h, n_walks, max_len_arr, max_len_cap, bias_arr, start_policy, seed, flags) -> TuneReport:
    rep = TuneReport()
    _check(h, load().tempest_autotune_mixed(h, int(n_walks), max_len_arr, int(max_len_cap), bias_arr,
                                            int(start_policy), int(seed) & ((1 << 64) - 1), int(flags),
                                            ctypes.byref(rep)))
    return rep


def tempest_autotune(h, n_walks, max_len, bias, start_policy, seed, flags) -> TuneReport:
    rep = TuneReport()
    _check(h, load().tempest_autotune(h, int(n_walks), int(max_len), int(bias), int(start_policy),
                                      int(seed) & ((1 << 64) - 1), int(flags), ctypes.byref(rep)))
    return rep


def tempest_last_walk_stats(h) -> WalkStats:
    ws = WalkStats()
    _check(h, load().tempest_last_walk_stats(h, ctypes.byref(ws)))
    return ws


def tempest_get_counts(h):
    out = (ctypes.c_int64 * 10)()
    _check(h, load().tempest_get_counts(h, out))
    return list(out)


def tempest_export_state(h, which: int, dst_ptr, cap: int) -> int:
    n = ctypes.c_int64()
    _check(h, load().tempest_export_state(h, int(which), ctypes.c_void_p(dst_ptr) if dst_ptr else None,
                                          int(cap), ctypes.byref(n)))
    return n.value


def tempest_sync(h):
    return _check(h, load().tempest_sync(h))


def tempest_last_error(h) -> str:
    m = load().tempest_last_error(h)
    return m.decode() if m else ""


def tempest_sort_batch_noalloc(src_ptr, dst_ptr, ts_ptr, n, out_src_ptr, out_dst_ptr, out_ts_ptr, stream_ptr):
    """Allocation-free batch sort for callers that cannot allocate device
    memory at run time (see include/tempest.h)."""
    return _check(None, load().tempest_sort_batch_noalloc(
        ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr), ctypes.c_void_p(ts_ptr), int(n),
        ctypes.c_void_p(out_src_ptr), ctypes.c_void_p(out_dst_ptr), ctypes.c_void_p(out_ts_ptr),
        ctypes.c_void_p(stream_ptr)))


# ---------------------------------------------------------------- wrapper
def _ptr(x, dtype: Optional[str] = None):
    """Raw pointer of a contiguous tensor / array, checking its element type
    (one of "int32", "int64", "uint8")."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if dtype is not None and str(x.dtype) != "torch." + dtype:
            raise TypeError("expected a %s tensor, got %s" % (dtype, x.dtype))
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if dtype is not None and x.dtype != np.dtype(dtype):
        raise TypeError("expected a %s array, got %s" % (dtype, x.dtype))
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data


class Engine:
    """A handle plus tensor-friendly calls.  Inputs may be CPU or CUDA
    tensors (or numpy arrays); outputs are allocated on `device`."""

    COUNT_KEYS = ("m", "G_tot", "n_nodes", "M", "Gn", "dropped_late", "evicted", "has_cutoff",
                  "cutoff", "seq_next")

    def __init__(self, window: int = 0, directed: bool = True, device: str = "cuda",
                 torch_allocator: bool = False, hbm_budget: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.h = tempest_create(window, directed)
        self.directed = directed
        self._cb = None
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        tempest_set_stream(self.h, st.cuda_stream)
        self.stream = st
        if torch_allocator or hbm_budget:
            self.use_torch_allocator(hbm_budget)

    def use_torch_allocator(self, budget: int = 0):
        torch = self.torch
        dev = self.device.index if self.device.index is not None else torch.cuda.current_device()
        stream = self.stream

        @ALLOC_FN
        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            except Exception:
                return None

        @RELEASE_FN
        def _release(ptr, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._cb = (_alloc, _release)
        tempest_set_allocator(self.h, _alloc, _release, None, int(budget))

    def close(self):
        if getattr(self, "h", None) is not None:
            tempest_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_bias_params(self, lambda_hop: float, lambda_start: float = 0.0):
        tempest_set_bias_params(self.h, lambda_hop, lambda_start)

    def set_scheduler(self, mode: int):
        tempest_set_scheduler(self.h, mode)

    def set_tuning(self, knob: int, value: int):
        tempest_set_tuning(self.h, knob, value)

    def get_tuning(self, knob: int) -> int:
        return tempest_get_tuning(self.h, knob)

    def set_weight_rate(self, lambda_w: float):
        """Rate of the weight-based sampler (TEMPEST_BIAS_EXP_WEIGHT); keeps group weights from now on."""
        _check(self.h, load().tempest_set_weight_rate(self.h, float(lambda_w)))

    def active_nodes(self, direction: int = 0) -> int:
        """Number of nodes with a live entry (in-entry when direction is 1): PER_NODE walk counts are
        multiples of it."""
        return tempest_active_nodes(self.h, direction)

    def set_node2vec(self, p: float, q: float):
        """Return / in-out parameters of Temporal Node2Vec walks (BIAS_NODE2VEC)."""
        _check(self.h, load().tempest_set_node2vec(self.h, float(p), float(q)))

    def enable_backward(self):
        """Keep the in-edge index that backward walks of a directed graph read."""
        tempest_enable_backward(self.h)

    def autotune(self, n_walks, max_len, bias=BIAS_EXP, start_policy=0, seed=0, forms=True,
                 per_ingest=False) -> dict:
        """Time candidate settings on the live index and keep the fastest; per_ingest charges every
        timed call the rebuild of the derived indexes (a workload with an ingest before each call)."""
        flags = (TUNE_FORMS if forms else 0) | (TUNE_PER_INGEST if per_ingest else 0)
        return tempest_autotune(self.h, n_walks, max_len, bias, start_policy, seed, flags).as_dict()

    def autotune_mixed(self, max_len_arr, bias_arr, max_len_cap=None, start_policy=0, seed=0, forms=True) -> dict:
        """Autotune on a mixed request's own per-walk lengths and biases."""
        n = int(max_len_arr.shape[0])
        assert bias_arr.shape[0] == n
        cap = int(max_len_cap) if max_len_cap is not None else int(max_len_arr.max().item())
        return tempest_autotune_mixed(self.h, n, _ptr(max_len_arr, "int32"), cap, _ptr(bias_arr, "uint8"),
                                      start_policy, seed, TUNE_FORMS if forms else 0).as_dict()

    def ingest(self, src, dst, ts) -> dict:
        n = int(src.shape[0])
        assert dst.shape[0] == n and ts.shape[0] == n
        return tempest_ingest(self.h, _ptr(src, "int32"), _ptr(dst, "int32"), _ptr(ts, "int64"), n).as_dict()

    def walks(self, n_walks: int, max_len: int, bias: int = BIAS_UNIFORM,
              start_policy: int = START_UNIFORM_EDGE, seed: int = 0, out=None, direction: int = 0):
        torch = self.torch
        if out is None:
            node = torch.empty((n_walks, max_len), dtype=torch.int32, device=self.device)
            ts = torch.empty((n_walks, max_len), dtype=torch.int64, device=self.device)
            ln = torch.empty((n_walks,), dtype=torch.int32, device=self.device)
        else:
            node, ts, ln = out
        fn = tempest_walks_backward if direction else tempest_walks
        fn(self.h, n_walks, max_len, bias, start_policy, seed, _ptr(node, "int32"), _ptr(ts, "int64"),
           _ptr(ln, "int32"))
        return node, ts, ln

    def walks_mixed(self, max_len_arr, bias_arr, start_policy: int = START_UNIFORM_EDGE, seed: int = 0,
                    max_len_cap: Optional[int] = None, out=None):
        torch = self.torch
        n = int(max_len_arr.shape[0])
        cap = int(max_len_cap if max_len_cap is not None else (int(max_len_arr.max()) if n else 2))
        if out is None:
            node = torch.empty((n, cap), dtype=torch.int32, device=self.device)
            ts = torch.empty((n, cap), dtype=torch.int64, device=self.device)
            ln = torch.empty((n,), dtype=torch.int32, device=self.device)
        else:
            node, ts, ln = out
        tempest_walks_mixed(self.h, n, _ptr(max_len_arr, "int32"), cap, _ptr(bias_arr, "uint8"), start_policy,
                            seed, _ptr(node, "int32"), _ptr(ts, "int64"), _ptr(ln, "int32"))
        return node, ts, ln

    def last_walk_stats(self) -> dict:
        return tempest_last_walk_stats(self.h).as_dict()

    def counts(self) -> dict:
        return dict(zip(self.COUNT_KEYS, tempest_get_counts(self.h)))

    def export(self, which: int):
        """One state array as a numpy array (host copy)."""
        n = tempest_export_state(self.h, which, None, 0)
        dt = np.int64 if which == STATE_TS else np.int32
        out = np.zeros(max(n, 1), dt)
        if n:
            tempest_export_state(self.h, which, out.ctypes.data, n)
        return out[:n]

    def state(self) -> dict:
        c = self.counts()
        return dict(counts=c, src=self.export(STATE_SRC), dst=self.export(STATE_DST),
                    ts=self.export(STATE_TS), ts_group_off=self.export(STATE_TS_GROUP_OFF),
                    node_off=self.export(STATE_NODE_OFF), node_order=self.export(STATE_NODE_ORDER),
                    node_group_off=self.export(STATE_NODE_GROUP_OFF),
                    node_gidx=self.export(STATE_NODE_GIDX))

    def sync(self):
        tempest_sync(self.h)
