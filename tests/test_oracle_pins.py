"""Pins of the oracle to what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: brute-force
Eq. 1 sums, brute-force modularity differences, the greedy property that
defines the decoupling filter, a from-scratch Eq. 3 rebuild, the generator's
own record of the edge set, closed forms, and exhaustive search on tiny graphs.
"""
import numpy as np
import pytest

from oracle import Oracle, decouple
from synth import (EdgeStream, csr_from_arcs, planted_partition, planted_stream,
                   random_batch, random_small_graph, uniform_u64)
from tests import brute


def _graphs(count=24, nmax=12):
    out = []
    for seed in range(count):
        directed = seed % 2 == 1
        n = 5 + seed % (nmax - 4)
        g = random_small_graph(n, 0.35, directed, wmax=5, seed=seed, self_loops=(seed % 3 == 0))
        if g.nnz:
            out.append((seed, g))
    return out


def _stream_states(g, seed, batches=6, **params):
    """Yield (oracle, edge stream) after create and after each batch."""
    o = Oracle(g, **params)
    st = EdgeStream.from_graph(g, seed)
    yield o, st
    for t in range(batches):
        m = len(st.keys)
        b = random_batch(st, 3, min(2, m), min(1, max(0, m - 2)), 4, seed * 131 + t)
        assert o.apply(b) == 0
        yield o, st


def _graph_of_stream(st):
    s, d = st.keys // st.n, st.keys % st.n
    return csr_from_arcs(st.n, s, d, st.wts, st.directed)


# --------------------------------------------------------------------- Eq. 1
def test_modularity_numerator_is_eq1_double_sum():
    """Qnum = gd*m^2*Q equals the O(n^2) double sum of Eq. 1 on the oracle's
    labels, after create and after every batch (directed and undirected,
    with self-loops)."""
    for seed, g in _graphs():
        for o, st in _stream_states(g, seed, batches=4, L=2):
            W = brute.dense(_graph_of_stream(st))
            m, q = o.scalars()
            assert m == sum(map(sum, W))
            assert q == brute.q_numerator(W, o.labels().tolist()), seed
            if m:
                assert abs(o.modularity() - q / (m * m)) <= 1e-12 * max(1.0, abs(q / (m * m)))


def test_modularity_with_rational_gamma():
    for seed, g in _graphs(8):
        o = Oracle(g, gamma_num=3, gamma_den=2, L=1)
        W = brute.dense(g)
        _, q = o.scalars()
        assert q == brute.q_numerator(W, o.labels().tolist(), gn=3, gd=2)


# --------------------------------------------------------------------- Eq. 2
@pytest.mark.parametrize("level", [0, 1])
def test_gain_equals_bruteforce_modularity_change(level):
    """The exact Eq. 2 gain of moving node v to community b equals
    gd*m^2*(Q_after - Q_before) recomputed from scratch, for every v and every
    other community b (adjacent or not), at level 0 and at level 1 (where the
    move relabels every ground vertex of the supernode)."""
    checked = 0
    for seed, g in _graphs(16, nmax=11):
        o = Oracle(g, L=2, M_static=1)
        if o.top < level:
            continue
        W = brute.dense(g)
        lab0 = o.labels().tolist()
        base = brute.q_numerator(W, lab0)
        chain = [o.level(q).par for q in range(level)]
        Lr = o.level(level)
        comms = sorted(set(lab0))
        for v in np.flatnonzero(Lr.alive).tolist():
            members = brute.ground_members(chain, level, v) if level else [v]
            a = int(Lr.lab[v])
            for b in comms:
                if b == a:
                    continue
                new = list(lab0)
                for u in members:
                    new[u] = b
                assert o.gain(level, v, b) == brute.q_numerator(W, new) - base
                checked += 1
    assert checked > 50


# --------------------------------------------------------------------- Decouple
def _greedy_property(v, src, dst, g, acc):
    """Sec. III-E: in (gain desc, node asc) order a candidate is accepted iff
    no earlier accepted candidate made its source an acceptor or its target an
    emitter; and no community ends up both emitter and acceptor."""
    order = sorted(range(len(v)), key=lambda k: (-g[k], v[k]))
    for pos, k in enumerate(order):
        blocked = any(acc[j] and (dst[j] == src[k] or src[j] == dst[k]) for j in order[:pos])
        if bool(acc[k]) == blocked:
            return False
    emit = {src[k] for k in range(len(v)) if acc[k]}
    accept = {dst[k] for k in range(len(v)) if acc[k]}
    return not (emit & accept)


def test_decouple_is_the_greedy_filter():
    for seed in range(40):
        cnt = 1 + seed * 3
        comms = 2 + seed % 9
        idx = np.arange(cnt)
        src = uniform_u64(seed, 1, idx, comms)
        dst = (src + 1 + uniform_u64(seed, 2, idx, comms - 1)) % comms
        v = np.random.default_rng(seed).permutation(cnt * 2)[:cnt]
        g = [int(x) for x in uniform_u64(seed, 3, idx, 4)]  # few values: many ties
        if seed % 4 == 0:
            g = [x * (1 << 90) + 7 for x in g]  # beyond 64 bits
        acc = decouple(v, src, dst, g)
        assert _greedy_property(v.tolist(), src.tolist(), dst.tolist(), g, acc.tolist()), seed


# --------------------------------------------------------------------- repair
def test_level0_matches_generator_edge_set():
    """Batch application (the first step of Algorithm 1) reproduces the generator's own
    record of the evolving edge set, including reweights and deletes."""
    for seed, g in _graphs(12):
        for o, st in _stream_states(g, seed, batches=6):
            rp, col, w = o.level_adj(0)
            got = brute.csr_dict(rp, col, w)
            want = brute.csr_dict(*[getattr(_graph_of_stream(st), k) for k in ("row_ptr", "col", "w")])
            assert got == want


def test_aggregate_levels_equal_eq3_rebuild():
    """After create and after every batch, every level r+1 equals the Eq. 3
    grouped sum of level r through pi_r, strengths equal row sums, and the
    community totals equal those of the level-0 labels."""
    for seed, g in _graphs(16):
        for o, st in _stream_states(g, seed, batches=5, L=3, M_static=3):
            T = o.top
            for r in range(T):
                rp, col, w = o.level_adj(r)
                src = np.repeat(np.arange(g.n), np.diff(rp))
                par = o.level(r).par
                want = brute.rebuild_level(g.n, src, col, w, par)
                assert brute.csr_dict(*o.level_adj(r + 1)) == want, (seed, r)
            for r in range(T + 1):
                rp, col, w = o.level_adj(r)
                L = o.level(r)
                ko = np.zeros(g.n, np.int64)
                ki = np.zeros(g.n, np.int64)
                src = np.repeat(np.arange(g.n), np.diff(rp))
                np.add.at(ko, src, w)
                np.add.at(ki, col, w)
                assert np.array_equal(ko, L.kout) and np.array_equal(ki, L.kin)
            lab = o.labels()
            rp, col, w = o.level_adj(0)
            src = np.repeat(np.arange(g.n), np.diff(rp))
            Ko, Ki, e = o.comm()
            assert np.array_equal(Ko, np.bincount(lab[src], weights=w, minlength=g.n).astype(np.int64))
            assert np.array_equal(Ki, np.bincount(lab[col], weights=w, minlength=g.n).astype(np.int64))
            inside = lab[src] == lab[col]
            assert np.array_equal(e, np.bincount(lab[src][inside], weights=w[inside],
                                                 minlength=g.n).astype(np.int64))
            assert o.check() == ""


def test_label_invariant_and_nesting():
    """P^r(u) = P^{r+1}(pi_r(u)) at every level; every refined community lies
    inside one community and is weakly connected in G^r."""
    for seed, g in _graphs(16):
        for o, st in _stream_states(g, seed, batches=4, L=3, M_static=4):
            for r in range(o.top):
                L, Ln = o.level(r), o.level(r + 1)
                rp, col, w = o.level_adj(r)
                src = np.repeat(np.arange(g.n), np.diff(rp))
                pairs = list(zip(src.tolist(), col.tolist()))
                alive = np.flatnonzero(L.alive)
                assert np.array_equal(L.lab[alive], Ln.lab[L.par[alive]])
                for x in np.unique(L.par[alive]):
                    members = alive[L.par[alive] == x].tolist()
                    assert brute.weakly_connected(members, pairs), (seed, r, x)


def test_delete_then_reinsert_restores_statistics():
    """With the update passes switched off (N=0), a batch followed by its
    inverse restores every array bit for bit (Eq. 3 linearity)."""
    for seed, g in _graphs(12):
        o = Oracle(g, N=0, L=3)
        before = _snapshot(o)
        st = EdgeStream.from_graph(g, seed)
        st0 = EdgeStream(st.n, st.directed, st.keys.copy(), st.wts.copy(), st.seed)
        m = len(st.keys)
        b = random_batch(st, 3, min(2, m), min(1, max(0, m - 2)), 4, seed)
        assert o.apply(b) == 0
        assert o.apply(brute.inverse_batch(b, st0)) == 0
        after = _snapshot(o)
        for k in before:
            assert np.array_equal(before[k], after[k]), (seed, k)


def _snapshot(o):
    out = {}
    for r in range(o.top + 1):
        L = o.level(r)
        for k in ("lab", "par", "kout", "kin", "cnt", "alive"):
            out[f"{k}{r}"] = getattr(L, k).copy()
        for k, a in zip(("rp", "col", "w"), o.level_adj(r)):
            out[f"{k}{r}"] = a
    for k, a in zip(("Kout", "Kin", "e"), o.comm()):
        out[k] = a
    out["scal"] = np.array(o.scalars(), dtype=object)
    return out


def test_undirected_equals_symmetric_directed():
    """An undirected graph and the same symmetric matrix run as a directed
    graph give identical partitions, hierarchies and modularity."""
    for seed in range(10):
        g = random_small_graph(10 + seed, 0.3, False, wmax=4, seed=seed)
        gd = csr_from_arcs(g.n, *g.arcs(), directed=True)
        ou, od = Oracle(g, L=3), Oracle(gd, L=3)
        st = EdgeStream.from_graph(g, seed)
        for t in range(5):
            assert ou.top == od.top
            for r in range(ou.top + 1):
                a, b = ou.level(r), od.level(r)
                for k in ("lab", "par", "kout", "kin", "cnt", "alive"):
                    assert np.array_equal(getattr(a, k), getattr(b, k)), (seed, t, r, k)
            assert ou.scalars() == od.scalars()
            m = len(st.keys)
            bu = random_batch(st, 2, min(2, m), min(1, max(0, m - 2)), 4, seed * 7 + t)
            # the directed run names both arcs of every undirected update
            fix = []
            for s, d, op, w in bu.tolist():
                fix.append([s, d, op, w])
                fix.append([d, s, op, w])
            assert ou.apply(bu) == 0
            assert od.apply(np.array(fix, dtype=np.int32)) == 0


# --------------------------------------------------------------------- passes
def test_batch_never_lowers_modularity():
    """Rollback of negative mini-batches makes Q_t(P_t) >= Q_t(P_{t-1}):
    the numerator after the passes is at least its value right after the
    statistic repair, for every batch."""
    g = planted_partition(n=2000, block=50, seed=5)
    o = Oracle(g)
    for b in planted_stream(g, batches=8, size=60, seed=5, block=50):
        assert o.apply(b) == 0
        assert o.scalars()[1] >= o.q_after_repair()


def test_empty_batch_changes_nothing():
    g = planted_partition(n=1000, block=50, seed=6)
    o = Oracle(g)
    s0 = _snapshot(o)
    assert o.apply(np.zeros((0, 4), np.int32)) == 0
    # a batch whose net change is zero
    s, d = int(g.arcs()[0][0]), int(g.arcs()[1][0])
    w = int(g.w[0])
    assert o.apply(np.array([[s, d, 2, w + 1], [s, d, 2, w]], np.int32)) == 0
    s1 = _snapshot(o)
    for k in s0:
        assert np.array_equal(s0[k], s1[k]), k


@pytest.mark.parametrize("bad,status", [
    ([[0, 10_000, 0, 1]], 2),      # vertex id out of range
    ([[-1, 3, 0, 1]], 2),
    ([[0, 1, 7, 1]], 1),           # unknown op
    ([[0, 1, 0, 0]], 1),           # insert of weight 0
    ([[0, 1, 2, -3]], 4),          # negative reweight
    ([[2, 999, 1, 0]], 3),         # delete of an absent edge
    ([[2, 999, 2, 5]], 3),         # reweight of an absent edge
    ([[5, 6, 0, 2**31 - 1], [5, 6, 0, 2**31 - 1]], 8),  # weight overflow
])
def test_invalid_batches_are_rejected_atomically(bad, status):
    g = planted_partition(n=1000, block=50, seed=7)
    o = Oracle(g)
    s0 = _snapshot(o)
    ok = [[1, 2, 0, 1]]
    assert o.apply(np.array(ok + bad, np.int32)) == status
    s1 = _snapshot(o)
    for k in s0:
        assert np.array_equal(s0[k], s1[k]), k


def test_first_failing_update_sets_the_status():
    g = planted_partition(n=1000, block=50, seed=7)
    o = Oracle(g)
    batch = np.array([[3, 998, 1, 0], [0, 1, 2, -1]], np.int32)  # NO_EDGE at 0, NEG at 1
    assert o.apply(batch) == 4  # single-update checks come first
    batch = np.array([[3, 998, 2, 1], [4, 997, 1, 0]], np.int32)
    assert o.apply(batch) == 3


def test_rerun_is_bit_identical():
    g = planted_partition(n=2000, block=50, seed=8)
    bs = planted_stream(g, batches=4, size=80, seed=8, block=50)
    runs = []
    for _ in range(2):
        o = Oracle(g)
        for b in bs:
            o.apply(b)
        runs.append(_snapshot(o))
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k])


# --------------------------------------------------------------------- static
@pytest.mark.parametrize("k,s", [(2, 3), (3, 4), (5, 5), (8, 3)])
def test_static_leiden_finds_disjoint_cliques(k, s):
    """k disjoint equal cliques: the optimum puts each clique in its own
    community with Q = 1 - 1/k exactly (Eq. 1 with e_C = K_C = s(s-1))."""
    src, dst = [], []
    for c in range(k):
        for i in range(s):
            for j in range(i + 1, s):
                src.append(c * s + i)
                dst.append(c * s + j)
    g = csr_from_arcs(k * s, src, dst, np.ones(len(src)), directed=False)
    o = Oracle(g)
    lab = o.labels()
    for c in range(k):
        assert len(set(lab[c * s:(c + 1) * s].tolist())) == 1
    assert len(set(lab.tolist())) == k
    m, q = o.scalars()
    assert q * k == (k - 1) * m * m  # Q = 1 - 1/k


def test_static_never_beats_bruteforce_optimum():
    for seed in range(10):
        g = random_small_graph(7 + seed % 3, 0.4, seed % 2 == 1, wmax=3, seed=100 + seed)
        if not g.nnz:
            continue
        W = brute.dense(g)
        best = max(brute.q_numerator(W, p) for p in brute.set_partitions(g.n))
        o = Oracle(g)
        _, q = o.scalars()
        assert q <= best
        assert q == brute.q_numerator(W, o.labels().tolist())


def test_planted_partition_is_recovered():
    """Sanity on the 10,000-vertex planted partition: static Leiden reaches
    at least the planted labels' modularity and recovers them (ARI)."""
    g = planted_partition()
    o = Oracle(g)
    W_q = o.modularity()
    s, d, w = g.arcs()
    lab = g.planted
    m = w.sum()
    ko = np.bincount(lab[s], weights=w)
    e = np.bincount(lab[s][lab[s] == lab[d]], weights=w[lab[s] == lab[d]])
    q_planted = (e / m - (ko / m) ** 2).sum()
    assert W_q >= 0.99 * q_planted  # a heuristic: close to, not always above
    assert brute.ari(o.labels(), lab) > 0.95


# --------------------------------------------------------------------- growth
@pytest.mark.parametrize("directed", [False, True])
def test_growth_keeps_every_invariant(directed):
    """Vertex-set growth (Sec. II): new isolated vertices leave the Eq. 1
    numerator unchanged, every invariant of the hierarchy (Eq. 3 rebuild,
    strengths, label and seed invariants, community totals) holds, and later
    batches that connect the new vertices keep it so; the numerator still
    equals the brute-force Eq. 1 sum on the grown graph."""
    for seed in range(6):
        g = random_small_graph(10 + seed, 0.3, directed, wmax=3, seed=600 + seed)
        if not g.nnz:
            continue
        o = Oracle(g, L=2, M_static=3)
        st = EdgeStream.from_graph(g, seed)
        b = random_batch(st, 3, 1, 1, 3, seed)
        assert o.apply(b) == 0
        m0, q0 = o.scalars()
        o.grow(g.n + 5)
        assert o.check() == ""
        assert o.scalars() == (m0, q0)
        assert (o.labels()[g.n:] == np.arange(g.n, g.n + 5)).all()
        st2 = EdgeStream(g.n + 5, st.directed, st.keys // st.n * (g.n + 5) + st.keys % st.n, st.wts, seed)
        for t in range(4):
            b = random_batch(st2, 4, 1, 1, 3, seed * 11 + t)
            assert o.apply(b) == 0
            assert o.check() == ""
            W = brute.dense(_graph_of_stream(st2))
            assert o.scalars()[1] == brute.q_numerator(W, o.labels().tolist())
