"""The largest stream's recipe (undirected R-MAT at scale 28, ids below
214,000,000, 3.30e9 distinct edges, unit weights, log-uniform batch sizes
with 70/20/10 inserts/deletes/reweights) at reduced scales: the graph has the
recipe's size and shape, the torch builder gives the numpy builder's graph
bit for bit, and every batch of the stream is valid against the edge set it
is applied to."""
import numpy as np
import pytest

from synth import DELETE, INSERT, REWEIGHT, c5_size, c5_stream, rmat_undirected_c5


def test_recipe_sizes():
    assert c5_size(0) == (214_000_000, 3_300_000_000, 28)
    assert c5_size(3) == (26_750_000, 412_500_000, 25)


def test_graph_shape_at_reduced_scale():
    g = rmat_undirected_c5(13)
    n, edges, _ = c5_size(13)
    assert g.n == n and not g.directed
    assert g.nnz == 2 * edges
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    col = g.col.astype(np.int64)
    assert (src != col).all() and col.max() < n
    assert (g.w == 1).all()
    fwd = np.sort(src * n + col)
    rev = np.sort(col * n + src)
    assert np.array_equal(fwd, rev)  # symmetric
    assert len(np.unique(fwd)) == len(fwd)  # distinct arcs
    for v in range(0, n, max(1, n // 64)):  # rows sorted
        r = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert (np.diff(r) > 0).all()
    deg = np.diff(g.row_ptr)
    assert deg.max() > 20 * deg.mean()  # R-MAT skew: hubs


def test_torch_builder_matches_numpy():
    torch = pytest.importorskip("torch")
    from synth.streams import rmat_undirected_c5_t
    g = rmat_undirected_c5(12)
    h = rmat_undirected_c5_t(12, device="cpu")
    assert np.array_equal(g.row_ptr, h.row_ptr) and np.array_equal(g.col, h.col)
    assert torch is not None


def test_stream_is_valid_against_the_edge_set():
    g = rmat_undirected_c5(12)
    bs = c5_stream(g, 30, max_size=20_000)
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    live = set((src * n + g.col).tolist())
    sizes = np.array([len(b) for b in bs])
    assert sizes.min() >= 10 and sizes.max() <= 20_000
    assert len(set(sizes.tolist())) > 20
    gone = set()
    for b in bs:
        s, d, op = b[:, 0].astype(np.int64), b[:, 1].astype(np.int64), b[:, 2]
        k = np.minimum(s, d) * n + np.maximum(s, d)
        assert (s != d).all() and s.max() < n and d.max() < n
        nd, nr = int((op == DELETE).sum()), int((op == REWEIGHT).sum())
        assert abs(nd - round(0.2 * len(b))) <= 1 and abs(nr - round(0.1 * len(b))) <= 1
        assert (b[op == REWEIGHT, 3] >= 1).all() and (b[op == INSERT, 3] >= 1).all()
        for kk in k[(op == DELETE) | (op == REWEIGHT)].tolist():
            a, c = divmod(kk, n)
            assert a * n + c in live and kk not in gone  # an existing edge, never deleted before
        for kk in k[op == DELETE].tolist():
            gone.add(kk)
            a, c = divmod(kk, n)
            live.discard(a * n + c)
            live.discard(c * n + a)
        for a, c in zip(s[op == INSERT].tolist(), d[op == INSERT].tolist()):
            live.add(a * n + c)
            live.add(c * n + a)
            gone.discard(min(a, c) * n + max(a, c))
