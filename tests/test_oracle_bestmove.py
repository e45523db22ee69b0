"""Pins of the oracle's BestMove and BestRef choices (CPU only).

The move loop and the refinement loop pick, per node, the target with the
largest positive exact gain among the admissible targets, ties going to the
lowest id.  These tests run the oracle's own best_move / best_ref (the very
functions its loops call) on one node at a time and compare the chosen
(target, gain) with an exhaustive search in which every gain is the change of
the Eq. 1 numerator recomputed from scratch (an O(n^2) double sum over the
ground graph) after relabelling the node's ground vertices:

  * BestMove (Eq. 2, Algorithm 1's move step): the admissible targets are the
    communities of the node's level-r neighbours other than its own; only a
    positive gain counts.  A non-adjacent community is never chosen, even
    when its brute-force gain is larger.
  * BestRef (the refinement step): the node is a singleton refined community;
    the admissible targets are the refined communities of its same-community
    level-r neighbours; the gain is the change of the numerator of the refined
    partition.

States come from static builds and update streams of random small graphs
(directed and undirected, gamma = 1 and 3/2) and, for BestMove, from random
partitions set directly on one-level states, which produce exact ties,
nodes without any positive move, and non-adjacent communities that beat every
adjacent one.
"""
import numpy as np
import pytest

from oracle import Oracle
from synth import EdgeStream, csr_from_arcs, random_batch, random_small_graph, uniform_u64
from tests import brute


def _ground(st):
    s, d = st.keys // st.n, st.keys % st.n
    return csr_from_arcs(st.n, s, d, st.wts, st.directed)


def _anc(o, r):
    """Level-r ancestor of every ground vertex, following the parent maps."""
    a = np.arange(o.n)
    for q in range(r):
        a = o.level(q).par[a]
    return a


def _neighbours(g, anc, x):
    """Level-r neighbours of node x (out and in, self excluded), built from the
    ground arcs mapped through the ancestors, not from the oracle's rows."""
    s, d, _ = g.arcs()
    out = set()
    for a, b in zip(anc[s].tolist(), anc[d].tolist()):
        if a == x and b != x:
            out.add(b)
        if b == x and a != x:
            out.add(a)
    return out


def _argmax(cands):
    """Largest positive gain, ties to the lowest id; None when none is positive."""
    best = None
    for t, gval in sorted(cands.items()):
        if gval > 0 and (best is None or gval > best[1]):
            best = (t, gval)
    return best


class Tally:
    def __init__(self):
        self.nodes = self.ties = self.none = self.nonadj_better = 0


def _check_best_move(o, g, r, gn, gd, tally):
    W = brute.dense(g)
    anc = _anc(o, r)
    lab0 = o.labels().tolist()
    base = brute.q_numerator(W, lab0, gn, gd)
    Lr = o.level(r)
    comms = sorted(set(lab0))
    for v in np.flatnonzero(Lr.alive).tolist():
        a = int(Lr.lab[v])
        members = np.flatnonzero(anc == v).tolist()
        gains = {}
        for c in comms:
            if c == a:
                continue
            new = list(lab0)
            for u in members:
                new[u] = c
            gains[c] = brute.q_numerator(W, new, gn, gd) - base
        adj = {int(Lr.lab[y]) for y in _neighbours(g, anc, v)} - {a}
        want = _argmax({c: gains[c] for c in adj})
        got = o.best_move(r, v)
        assert got == want, (r, v, got, want)
        tally.nodes += 1
        pos = [gains[c] for c in adj if gains[c] > 0]
        if want is not None and pos.count(want[1]) > 1:
            tally.ties += 1
        if want is None:
            tally.none += 1
        top_non = max((gains[c] for c in comms if c != a and c not in adj), default=None)
        if top_non is not None and top_non > 0 and (want is None or top_non > want[1]):
            tally.nonadj_better += 1


def _check_best_ref(o, g, r, gn, gd, tally):
    W = brute.dense(g)
    anc = _anc(o, r)
    Lr, Ln = o.level(r), o.level(r + 1)
    ref0 = Lr.par[anc].tolist()  # refined id of every ground vertex
    base = brute.q_numerator(W, ref0, gn, gd)
    for v in np.flatnonzero(Lr.alive).tolist():
        if Lr.par[v] != v or Ln.cnt[v] != 1:
            continue
        members = np.flatnonzero(anc == v).tolist()
        cands = {}
        for y in _neighbours(g, anc, v):
            if Lr.lab[y] != Lr.lab[v]:
                continue
            X = int(Lr.par[y])
            if X == v or X in cands:
                continue
            new = list(ref0)
            for u in members:
                new[u] = X
            cands[X] = brute.q_numerator(W, new, gn, gd) - base
        want = _argmax(cands)
        got = o.best_ref(r, v)
        assert got == want, (r, v, got, want)
        tally.nodes += 1
        if want is None:
            tally.none += 1
        elif list(cands.values()).count(want[1]) > 1:
            tally.ties += 1


def _states(seed, directed, gn, gd, batches, **params):
    g = random_small_graph(7 + seed % 6, 0.35, directed, wmax=3 if seed % 2 else 1, seed=seed,
                           self_loops=seed % 3 == 0)
    if not g.nnz:
        return
    o = Oracle(g, gamma_num=gn, gamma_den=gd, **params)
    st = EdgeStream.from_graph(g, seed)
    yield o, _ground(st)
    for t in range(batches):
        m = len(st.keys)
        b = random_batch(st, 3, min(2, m), min(1, max(0, m - 2)), 3, seed * 71 + t)
        assert o.apply(b) == 0
        yield o, _ground(st)


@pytest.mark.parametrize("gamma", [(1, 1), (3, 2)])
@pytest.mark.parametrize("directed", [False, True])
def test_best_move_is_the_bruteforce_argmax(directed, gamma):
    """Static builds and update streams: BestMove at every level that exists."""
    gn, gd = gamma
    t = Tally()
    levels = set()
    for seed in range(14):
        for o, g in _states(seed, directed, gn, gd, 3, L=2, M_static=1, M=2):
            for r in range(o.top + 1):
                _check_best_move(o, g, r, gn, gd, t)
                levels.add(r)
    assert t.nodes > 200 and levels >= {0, 1}
    assert t.none > 0 and t.nodes - t.none > 10


@pytest.mark.parametrize("gamma", [(1, 1), (3, 2)])
@pytest.mark.parametrize("directed", [False, True])
def test_best_move_on_set_partitions(directed, gamma):
    """Random partitions set on one-level states: exact ties (unit weights),
    nodes with no positive move, and non-adjacent communities whose gain beats
    every adjacent one, which must not be chosen (at gamma = 1 in an undirected
    graph this needs a self-loop on the node: it adds to the node's strength
    but to no w(v, b))."""
    gn, gd = gamma
    t = Tally()
    for seed in range(24):
        g = random_small_graph(8 + seed % 5, 0.3, directed, wmax=1 if seed % 2 == 0 else 4, seed=100 + seed,
                               self_loops=seed % 3 != 2)
        if not g.nnz:
            continue
        o = Oracle(g, gamma_num=gn, gamma_den=gd, L=0)
        for trial in range(3):
            k = 2 + (seed + trial) % 5
            lab = uniform_u64(seed, 40 + trial, np.arange(g.n), k).astype(np.int64) * (g.n // k)
            o.set_partition(lab)
            assert o.check() == ""
            _check_best_move(o, g, 0, gn, gd, t)
    assert t.nodes > 300
    assert t.ties > 0 and t.none > 0 and t.nonadj_better > 0


@pytest.mark.parametrize("gamma", [(1, 1), (3, 2)])
@pytest.mark.parametrize("directed", [False, True])
def test_best_ref_is_the_bruteforce_argmax(directed, gamma):
    """Every singleton refined community at every refined level, after static
    builds that stop refinement early (M_static = 1) and after updates."""
    gn, gd = gamma
    t = Tally()
    for seed in range(20):
        for o, g in _states(seed, directed, gn, gd, 3, L=2, M_static=1, M=1):
            for r in range(o.top):
                _check_best_ref(o, g, r, gn, gd, t)
    assert t.nodes > 40
    assert t.none > 0 and t.nodes - t.none > 5
