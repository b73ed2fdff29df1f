"""Helpers that compare the CUDA library with the oracle."""
import numpy as np

STATE_KEYS = ("src", "dst", "ts", "ts_group_off", "node_off", "node_order", "node_group_off", "node_gidx")
COUNT_KEYS = ("m", "G_tot", "n_nodes", "M", "Gn", "dropped_late", "evicted", "has_cutoff", "seq_next")

# Biased walks: at least this fraction of hops must agree, and a walk may
# first diverge only at a draw whose oracle value x lies within BOUND_UNITS
# error bounds of an integer.  The oracle reports each draw's distance to the
# nearest integer in units of the double evaluation's own rounding bound
# (a few ulps of x plus the one-ulp error of exp / log carried through the
# formula, orc_sampler_x_bound); two evaluations that each stay within that
# bound can floor to different indexes only within twice it.  A GPU draw
# decided in FP32 on a bound that is too small shows up as a divergence many
# units away.
MIN_HOP_AGREEMENT = 0.9999
BOUND_UNITS = 2.0


def assert_state_equal(gpu: dict, orc: dict, where=""):
    for k in COUNT_KEYS:
        assert gpu["counts"][k] == orc["counts"][k], "%s count %s: gpu %r oracle %r" % (
            where, k, gpu["counts"][k], orc["counts"][k])
    if orc["counts"]["has_cutoff"]:
        assert gpu["counts"]["cutoff"] == orc["counts"]["cutoff"], where
    for k in STATE_KEYS:
        a = np.asarray(gpu[k]).astype(np.int64)
        b = np.asarray(orc[k]).astype(np.int64)
        assert a.shape == b.shape, "%s %s shape gpu %s oracle %s" % (where, k, a.shape, b.shape)
        if not np.array_equal(a, b):
            i = int(np.nonzero(a != b)[0][0])
            raise AssertionError("%s %s differs first at %d: gpu %d oracle %d" % (where, k, i, a[i], b[i]))


def assert_walks_bit_exact(g, o, where=""):
    gn, gt, gl = (np.asarray(x) for x in g)
    on, ot, ol = o[0], o[1], o[2]
    assert gl.shape == ol.shape
    if not np.array_equal(gl, ol):
        i = int(np.nonzero(gl != ol)[0][0])
        raise AssertionError("%s len differs at walk %d: gpu %d oracle %d" % (where, i, gl[i], ol[i]))
    for name, a, b in (("node", gn, on), ("ts", gt, ot)):
        if not np.array_equal(a, b):
            w, p = (int(x[0]) for x in np.nonzero(a != b))
            raise AssertionError("%s %s differs at walk %d pos %d: gpu %d oracle %d" % (
                where, name, w, p, a[w, p], b[w, p]))


def compare_biased(g, o, margin):
    """Returns (agreeing hops, total hops, divergences) and checks that every
    divergence sits at a sampler boundary."""
    gn, gt, gl = (np.asarray(x) for x in g)
    on, ot, ol = o[0], o[1], o[2]
    hops_total = int(np.clip(ol - 1, 0, None).sum())
    same = (gn == on).all(1) & (gt == ot).all(1) & (gl == ol)
    agree = int(np.clip(ol[same] - 1, 0, None).sum())
    div = []
    for w in np.nonzero(~same)[0]:
        diff = np.nonzero((gn[w] != on[w]) | (gt[w] != ot[w]))[0]
        p = int(diff[0]) if diff.size else int(min(gl[w], ol[w]))
        q = max(p, 1)
        mg = margin[w, q] if q < margin.shape[1] else np.inf
        assert mg <= BOUND_UNITS, "walk %d diverges at pos %d away from a boundary (margin %g bounds)" % (
            w, p, mg)
        agree += max(0, q - 1)
        div.append((int(w), p, float(mg)))
    return agree, hops_total, div
