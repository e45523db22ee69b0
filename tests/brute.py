"""Brute-force references used to pin the oracle (plain Python/numpy, tiny inputs).

None of this shares code with the oracle or with the CUDA library: modularity
is summed over every ordered vertex pair exactly as Eq. 1 is written, and
aggregate levels are rebuilt from the ground graph with numpy grouping.
"""
from __future__ import annotations

import itertools

import numpy as np


def dense(g):
    """Weight matrix of a CSR graph (Python ints)."""
    W = [[0] * g.n for _ in range(g.n)]
    s, d, w = g.arcs()
    for a, b, x in zip(s.tolist(), d.tolist(), w.tolist()):
        W[a][b] += x
    return W


def q_numerator(W, labels, gn=1, gd=1):
    """gd*m^2*Q from Eq. 1 as the double sum over all ordered pairs (i, j):
    Q = (1/m) sum_ij (w_ij - gamma k_i^out k_j^in / m) [c_i = c_j]."""
    n = len(W)
    m = sum(sum(row) for row in W)
    kout = [sum(W[i]) for i in range(n)]
    kin = [sum(W[i][j] for i in range(n)) for j in range(n)]
    tot = 0
    for i in range(n):
        for j in range(n):
            if labels[i] == labels[j]:
                tot += gd * m * W[i][j] - gn * kout[i] * kin[j]
    return tot


def set_partitions(n):
    """All set partitions of range(n) as label lists (restricted growth strings)."""
    def rec(i, labels, k):
        if i == n:
            yield list(labels)
            return
        for c in range(k + 1):
            labels.append(c)
            yield from rec(i + 1, labels, max(k, c + 1))
            labels.pop()
    yield from rec(0, [], 0)


def ground_members(par_chain, r, x):
    """Ground vertices represented by level-r node x, following parents up."""
    n = len(par_chain[0]) if par_chain else 0
    out = []
    for v in range(n):
        y = v
        for q in range(r):
            y = int(par_chain[q][y])
        if y == x:
            out.append(v)
    return out


def rebuild_level(n, src, dst, w, par):
    """Eq. 3: aggregate arcs of one level through the parent map; returns a
    dict {(x, y): weight} without zero entries."""
    out = {}
    for a, b, x in zip(src.tolist(), dst.tolist(), w.tolist()):
        key = (int(par[a]), int(par[b]))
        out[key] = out.get(key, 0) + int(x)
    return {k: v for k, v in out.items() if v != 0}


def csr_dict(rp, col, w):
    out = {}
    for v in range(len(rp) - 1):
        for k in range(rp[v], rp[v + 1]):
            out[(v, int(col[k]))] = int(w[k])
    return out


def weakly_connected(nodes, adj_pairs):
    """True when the subgraph induced by `nodes` is weakly connected."""
    nodes = set(nodes)
    if len(nodes) <= 1:
        return True
    nb = {v: set() for v in nodes}
    for a, b in adj_pairs:
        if a in nodes and b in nodes and a != b:
            nb[a].add(b)
            nb[b].add(a)
    start = next(iter(nodes))
    seen = {start}
    stack = [start]
    while stack:
        v = stack.pop()
        for u in nb[v]:
            if u not in seen:
                seen.add(u)
                stack.append(u)
    return seen == nodes


def ari(a, b):
    """Adjusted Rand index of two labelings."""
    a = np.asarray(a)
    b = np.asarray(b)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    cont = np.zeros((ai.max() + 1, bi.max() + 1), dtype=np.int64)
    np.add.at(cont, (ai, bi), 1)

    def c2(x):
        return x * (x - 1) / 2.0
    s = c2(cont).sum()
    sa = c2(cont.sum(1)).sum()
    sb = c2(cont.sum(0)).sum()
    exp = sa * sb / c2(len(a))
    mx = (sa + sb) / 2.0
    return float((s - exp) / (mx - exp)) if mx != exp else 1.0


def inverse_batch(batch, stream_before):
    """Batch that undoes `batch` given the edge set before it."""
    n = stream_before.n
    out = []
    for s, d, op, w in reversed(batch.tolist()):
        k = stream_before.canon(np.array([s]), np.array([d]))[0]
        pos = np.searchsorted(stream_before.keys, k)
        old = int(stream_before.wts[pos]) if pos < len(stream_before.keys) and stream_before.keys[pos] == k else 0
        if op == 0:
            out.append([s, d, 1, 0] if old == 0 else [s, d, 2, old])
        elif op == 1:
            out.append([s, d, 0, old])
        else:
            out.append([s, d, 2, old])
    return np.array(out, dtype=np.int32).reshape(-1, 4)


def all_pairs_product(n):
    return itertools.product(range(n), range(n))
