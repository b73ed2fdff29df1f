"""Brute-force restatements used to pin the oracle on tiny inputs.

These are written from the paper's set definitions, not from the oracle's
procedure: the live set is the window set W(t) of Sec. 2.6 filtered from all
non-late edges; the views of Sec. 2.3 are read off sorted tuples; Gamma_t(v)
of Sec. 2.1 is a filter over the live set; walk probabilities are products of
per-hop probabilities from the bias weights of Sec. 2.5.
"""
from __future__ import annotations

import math
from fractions import Fraction


def window_state(batches, window, directed):
    """Live set and views after each batch, by definition.

    Returns a list of dicts (one per batch)."""
    kept = []          # every non-late edge so far: (ts, seq, src, dst)
    cutoff = None
    seq = 0
    n_nodes = 0
    dropped = 0
    out = []
    for src, dst, ts in batches:
        for i in range(len(src)):
            n_nodes = max(n_nodes, src[i] + 1, dst[i] + 1)
            if cutoff is not None and ts[i] < cutoff:
                dropped += 1          # late: older than the cut-off in force
            else:
                kept.append((ts[i], seq + i, src[i], dst[i]))
        seq += len(src)
        if kept:
            tmax = max(e[0] for e in kept)
            if window > 0:
                c = tmax - window
                cutoff = c if cutoff is None else max(cutoff, c)
            elif window < 0:
                W = -window
                newest = sorted(kept, reverse=True)
                if len(newest) > W:
                    c = newest[W - 1][0]   # timestamp of the W-th newest edge
                    cutoff = c if cutoff is None else max(cutoff, c)
        live = sorted(e for e in kept if cutoff is None or e[0] >= cutoff)
        evicted = len(kept) - len(live)
        m = len(live)
        ts_group_off = [i for i in range(m) if i == 0 or live[i][0] != live[i - 1][0]] + [m]
        # node view: (node, ts, seq, side) order
        ent = []
        for p, (t, s, a, b) in enumerate(live):
            if directed:
                ent.append((a, t, s, 0, p))
            else:
                ent.append((a, t, s, 0, 2 * p))
                ent.append((b, t, s, 1, 2 * p + 1))
        ent.sort()
        node_order = [e[4] for e in ent]
        node_off = [sum(1 for e in ent if e[0] < v) for v in range(n_nodes + 1)]
        node_group_off = []
        node_gidx = []
        for v in range(n_nodes):
            node_gidx.append(len(node_group_off))
            seg = range(node_off[v], node_off[v + 1])
            for i in seg:
                if i == node_off[v] or ent[i][1] != ent[i - 1][1]:
                    node_group_off.append(i)
        node_gidx.append(len(node_group_off))
        node_group_off.append(len(ent))
        out.append(dict(src=[e[2] for e in live], dst=[e[3] for e in live], ts=[e[0] for e in live],
                        ts_group_off=ts_group_off, node_off=node_off, node_order=node_order,
                        node_group_off=node_group_off, node_gidx=node_gidx,
                        dropped_late=dropped, evicted=evicted_total(out, evicted),
                        cutoff=cutoff, n_nodes=n_nodes, live=live))
        kept = live[:]  # evicted edges never return
    return out


def evicted_total(prev, ev):
    return (prev[-1]["evicted"] if prev else 0) + ev


def group_weights(n, bias, lam):
    """Unnormalised weights of index i in [0, n) (Sec. 2.5)."""
    if bias == 0:
        return [1.0] * n
    if bias == 1:
        return [float(i + 1) for i in range(n)]
    return [math.exp(lam * i) for i in range(n)]


def gamma(live, directed, v, t):
    """Gamma_t(v): (other endpoint, ts) of live entries at v with ts > t, in
    (ts, seq, side) order (Sec. 2.1)."""
    g = []
    for (ts, seq, a, b) in live:
        if directed:
            if a == v and ts > t:
                g.append((ts, seq, 0, b))
        else:
            if a == v and ts > t:
                g.append((ts, seq, 0, b))
            if b == v and ts > t:
                g.append((ts, seq, 1, a))
    g.sort()
    return [(e[3], e[0]) for e in g]


def hop_distribution(live, directed, v, t, bias, lam, lam_w=None):
    """{(other, ts): probability} of the next hop, or {} when Gamma is empty.
    Bias 3 (weight-based): every edge of Gamma weighs exp(lam_w (ts - t_min))."""
    g = gamma(live, directed, v, t)
    if not g:
        return {}
    dist = {}
    if bias == 3:
        t_min = min(ts for _, ts in g)
        w = [math.exp(lam_w * (ts - t_min)) for _, ts in g]
        tot = sum(w)
        for e, x in zip(g, w):
            dist[e] = dist.get(e, 0.0) + x / tot
        return dist
    if bias == 0:
        for e in g:
            dist[e] = dist.get(e, 0.0) + 1.0 / len(g)
        return dist
    groups = sorted(set(ts for _, ts in g))
    w = group_weights(len(groups), bias, lam)
    tot = sum(w)
    for gi, gts in enumerate(groups):
        members = [e for e in g if e[1] == gts]
        for e in members:
            dist[e] = dist.get(e, 0.0) + w[gi] / tot / len(members)
    return dist


def node2vec_hop_distribution(live, directed, v, t, prev, lam, p, q):
    """Temporal Node2Vec (Sec. 2.5): the exponential proposal of
    hop_distribution reweighted by beta(prev, w) = 1/p (w == prev), 1 (a live
    edge prev -> w; either orientation when undirected), 1/q otherwise, then
    normalised: the law of rejection sampling on that proposal with accept
    probability beta / max(1/p, 1, 1/q).  prev None: the proposal itself."""
    d = hop_distribution(live, directed, v, t, 2, lam)
    if prev is None or not d:
        return d

    def adjacent(a, b):
        for (_, _, x, y) in live:
            if (x, y) == (a, b) or (not directed and (y, x) == (a, b)):
                return True
        return False

    out = {}
    for (w, ts), pr in d.items():
        beta = 1.0 / p if w == prev else (1.0 if adjacent(prev, w) else 1.0 / q)
        out[(w, ts)] = pr * beta
    tot = sum(out.values())
    return {k: x / tot for k, x in out.items()}


def start_distribution(live, directed, policy, bias, lam_start):
    """{(first node, second node, ts): probability} of the start edge."""
    m = len(live)
    dist = {}
    if m == 0:
        return dist
    if policy == 0:
        probs = [1.0 / m] * m
    else:
        groups = sorted(set(e[0] for e in live))
        w = group_weights(len(groups), bias, lam_start)
        tot = sum(w)
        probs = []
        for (ts, seq, a, b) in live:
            gi = groups.index(ts)
            size = sum(1 for e in live if e[0] == ts)
            probs.append(w[gi] / tot / size)
    for p, (ts, seq, a, b) in zip(probs, live):
        if directed:
            key = (a, b, ts)
            dist[key] = dist.get(key, 0.0) + p
        else:
            for key in ((a, b, ts), (b, a, ts)):
                dist[key] = dist.get(key, 0.0) + p / 2
    return dist


def walk_distribution(live, directed, max_len, bias, policy, lam_hop, lam_start, start_node=None, lam_w=None,
                      n2v=None):
    """Exact probability of every complete walk (tuple of (node, ts) pairs).
    With start_node the walk starts at that node and its first hop may take
    any of the node's live edges (the per-node start policy).  Bias 4 is
    Temporal Node2Vec with n2v = (p, q)."""
    out = {}

    def rec(path, p):
        v, t = path[-1]
        if t is None:
            t = float("-inf")
        if len(path) >= max_len:
            out[tuple(path)] = out.get(tuple(path), 0.0) + p
            return
        if bias == 4:
            prev = path[-2][0] if len(path) >= 2 else None
            d = node2vec_hop_distribution(live, directed, v, t, prev, lam_hop, *n2v)
        else:
            d = hop_distribution(live, directed, v, t, bias, lam_hop, lam_w)
        if not d:
            out[tuple(path)] = out.get(tuple(path), 0.0) + p
            return
        for (w, ts), q in d.items():
            rec(path + [(w, ts)], p * q)

    if start_node is not None:
        rec([(start_node, None)], 1.0)
        return out
    sb = 2 if bias in (3, 4) else bias  # weight-based and Node2Vec start like the index-based exponential
    for (a, b, ts), p in start_distribution(live, directed, policy, sb, lam_start).items():
        rec([(a, None), (b, ts)], p)
    return out


def cdf_exact(i, n, bias, lam=1.0):
    """P(index <= i) for the weights of Sec. 2.5, exactly (Fraction) for
    uniform / linear; as a high-precision Decimal for exponential."""
    if bias == 0:
        return Fraction(i + 1, n)
    if bias == 1:
        return Fraction((i + 1) * (i + 2), n * (n + 1))
    from decimal import Decimal, getcontext
    getcontext().prec = 80
    L = Decimal(lam)
    # sum_{j<=i} e^{L j} / sum_{j<n} e^{L j}, both geometric series
    num = (L * (i + 1)).exp() - 1
    den = (L * n).exp() - 1
    return num / den
