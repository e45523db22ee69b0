"""GPU unit tests through the C ABI (GB300 only): the device decoupling filter
against the oracle's on explicit candidate sets, the hierarchy returned in
ldl_result, and update streams at a rational resolution gamma = 3/2.
"""
import numpy as np
import pytest

from oracle import Oracle, decouple as oracle_decouple
from synth import EdgeStream, csr_from_arcs, planted_partition, planted_stream, random_batch, random_small_graph, \
    uniform_u64
from tests.parity import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ldl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2502_18497_gb300 import ldl as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def host_ctx(ldl):
    """A context with 2^16 node ids whose scratch the decoupling hook uses."""
    n = 1 << 16
    src = np.arange(0, 64, dtype=np.int64)
    g = csr_from_arcs(n, src, src + 1, np.ones(64, np.int64), directed=False)
    return ldl.LDL.from_graph(g)


def _candidates(seed, count, comms, gain_levels, big=False):
    idx = np.arange(count)
    v = np.random.default_rng(seed).permutation(1 << 16)[:count].astype(np.int32)
    src = uniform_u64(seed, 1, idx, comms).astype(np.int64)
    dst = uniform_u64(seed, 2, idx, comms - 1).astype(np.int64)
    dst = np.where(dst >= src, dst + 1, dst)  # dst != src
    g = uniform_u64(seed, 3, idx, gain_levels).astype(np.int64) + 1
    gains = [int(x) << 70 if big else int(x) for x in g.tolist()]
    if big:  # a few distinct low words so that the 128-bit order matters
        gains = [x + (k % 3) for k, x in enumerate(gains)]
    return v, src.astype(np.int32), dst.astype(np.int32), gains


@pytest.mark.parametrize("count,comms,levels,big", [
    (1, 2, 1, False), (37, 3, 2, False), (500, 5, 3, False), (4000, 40, 4, False),
    (3000, 10, 2, True), (8192, 300, 5, False), (8193, 300, 5, False), (20000, 2000, 3, False),
    (30000, 50, 2, True),
])
def test_decoupler_equals_the_serial_greedy(ldl, host_ctx, count, comms, levels, big):
    """Sec. III-E filter: the device rounds (one block up to 8192 candidates,
    the cooperative grid above) accept exactly the candidates the oracle's
    serial greedy accepts, on tie-heavy sets (few gain values, few
    communities) and with gains above 2^64."""
    for seed in range(3):
        v, src, dst, gains = _candidates(seed * 31 + count, count, comms, levels, big)
        want = oracle_decouple(v, src, dst, gains, id_space=1 << 16)
        got = host_ctx.debug_decouple(v, src, dst, gains)
        assert np.array_equal(got, want), (count, comms, seed, int(np.sum(got != want)))
        assert want.sum() > 0


def test_result_carries_the_hierarchy(ldl):
    """ldl_result returns H_t: per level the parent map, the community labels,
    the refined ids (the parent map) and node existence, on the device, equal
    to the state read back through ldl_get_level and to the oracle's."""
    g = planted_partition(n=3000, block=50, seed=21)
    o = Oracle(g)
    d = ldl.LDL.from_graph(g)
    for t, b in enumerate(planted_stream(g, batches=3, size=80, seed=21, block=50)):
        assert o.apply(b) == 0
        d.apply(b)
        h = d.hierarchy()
        assert len(h) == o.top + 1 == d.levels
        for r, lv in enumerate(h):
            lo = o.level(r)
            al = lo.alive.astype(bool)
            assert np.array_equal(lv["alive"], lo.alive)
            assert np.array_equal(lv["comm"][al], lo.lab[al])
            assert np.array_equal(lv["parent"][al], lo.par[al])
            assert np.array_equal(lv["refined"], lv["parent"])
            if r == o.top:
                assert (lv["parent"] == -1).all()
            assert np.array_equal(lv["parent"][~al], np.full(int((~al).sum()), -1, np.int32))


@pytest.mark.parametrize("directed", [False, True])
def test_random_streams_rational_gamma(ldl, directed):
    """Update streams at gamma = 3/2 (Eq. 1's resolution as gn/gd): the whole
    state equals the oracle's after creation and after every batch."""
    for seed in range(6):
        g = random_small_graph(24 + 9 * seed, 0.2, directed, wmax=4, seed=300 + seed, self_loops=seed % 2 == 1)
        if not g.nnz:
            continue
        params = dict(gamma_num=3, gamma_den=2, L=1 + seed % 4, M_static=3 + seed % 5, M=1 + seed % 5,
                      N=1 + seed % 3)
        o = Oracle(g, **params)
        d = ldl.LDL.from_graph(g, **params)
        msgs = compare_states(o, d, f"seed {seed} create")
        assert not msgs, "\n".join(msgs[:8])
        st = EdgeStream.from_graph(g, seed)
        for t in range(8):
            m = len(st.keys)
            b = random_batch(st, 5, min(3, m), min(2, max(0, m - 3)), 4, seed * 53 + t)
            assert o.apply(b) == 0
            d.apply(b)
            msgs = compare_states(o, d, f"seed {seed} batch {t}")
            assert not msgs, "\n".join(msgs[:8])


@pytest.mark.parametrize("directed", [False, True])
def test_planted_stream_rational_gamma(ldl, directed):
    """A 4,000-vertex planted partition (undirected) or R-MAT graph
    (directed) at gamma = 3/2, static build plus 5 batches."""
    from synth import rmat_directed, rmat_stream
    if directed:
        g = rmat_directed(scale=12, arcs=1 << 16, seed=77)
        bs = rmat_stream(g, batches=5, size=400, seed=77)
    else:
        g = planted_partition(n=4000, block=50, seed=77)
        bs = planted_stream(g, batches=5, size=120, seed=77, block=50)
    o = Oracle(g, gamma_num=3, gamma_den=2)
    d = ldl.LDL.from_graph(g, gamma_num=3, gamma_den=2)
    msgs = compare_states(o, d, "create")
    assert not msgs, "\n".join(msgs[:8])
    for t, b in enumerate(bs):
        assert o.apply(b) == 0
        d.apply(b)
        msgs = compare_states(o, d, f"batch {t}")
        assert not msgs, "\n".join(msgs[:8])


@pytest.mark.parametrize("directed", [False, True])
def test_random_streams_with_huge_weights(ldl, directed):
    """Weights up to 2^30 make m^2 far larger than 2^62, so the sweeps take
    their int128 gain path (small totals take the int64 one): the whole state
    still equals the oracle's after creation and every batch."""
    for seed in range(4):
        g = random_small_graph(30 + 7 * seed, 0.2, directed, wmax=1 << 30, seed=700 + seed)
        if not g.nnz:
            continue
        params = dict(L=2 + seed % 3, M_static=5, M=3, N=2)
        o = Oracle(g, **params)
        d = ldl.LDL.from_graph(g, **params)
        assert 6 * d.numerator()[0] ** 2 >= 1 << 62
        msgs = compare_states(o, d, f"seed {seed} create")
        assert not msgs, "\n".join(msgs[:8])
        st = EdgeStream.from_graph(g, seed)
        for t in range(6):
            m = len(st.keys)
            b = random_batch(st, 5, min(3, m), min(2, max(0, m - 3)), 1 << 30, seed * 31 + t)
            assert o.apply(b) == 0
            d.apply(b)
            msgs = compare_states(o, d, f"seed {seed} batch {t}")
            assert not msgs, "\n".join(msgs[:8])


@pytest.mark.parametrize("directed", [False, True])
def test_streams_without_rollback_match(ldl, directed):
    """ldl_params.no_rollback = 1 (no batch snapshot, no undo log) changes no
    result: the state equals the oracle's after every batch, and the batch
    estimate of such a context carries no snapshot."""
    from synth import rmat_directed, rmat_stream
    if directed:
        g = rmat_directed(scale=12, arcs=1 << 16, seed=91)
        bs = rmat_stream(g, batches=5, size=600, seed=91)
    else:
        g = planted_partition(n=4000, block=50, seed=91)
        bs = planted_stream(g, batches=5, size=150, seed=91, block=50)
    o = Oracle(g)
    d = ldl.LDL.from_graph(g, no_rollback=1)
    import ctypes
    est = ctypes.c_int64()
    assert ldl.load().ldl_batch_estimate_bytes(d._h, 150, ctypes.byref(est)) == 0 and est.value >= 0
    for t, b in enumerate(bs):
        assert o.apply(b) == 0
        d.apply(b)
        msgs = compare_states(o, d, f"batch {t}")
        assert not msgs, "\n".join(msgs[:8])


@pytest.mark.parametrize("count,bits,dup", [
    (0, 40, 1), (1, 40, 1), (2, 8, 1), (300, 16, 7), (2047, 40, 1), (2048, 40, 3), (2049, 40, 1),
    (5000, 9, 50), (6144, 40, 2), (6145, 40, 1), (40000, 40, 4), (49152, 40, 3), (49153, 33, 1),
    (300000, 40, 8), (1_300_000, 40, 2), (2_500_000, 44, 16),
])
def test_device_sort_is_a_stable_sort(ldl, host_ctx, count, bits, dup):
    """The device radix sort (one block up to 2048 pairs, one 8-block cluster
    up to 49152, one cooperative launch up to a few hundred tiles, separate
    launches per pass above) puts
    the pairs in the order of a stable sort by the low `bits` key bits:
    values carry each pair's input position, so equal keys must keep their
    input order.  Keys repeat (each drawn `dup`-fold on average) and some
    are skewed to one digit, as aggregate records are."""
    rng = np.random.default_rng(count * 7 + bits)
    distinct = max(1, count // dup)
    pool = rng.integers(0, 1 << bits, size=distinct, dtype=np.uint64) if bits < 64 else \
        rng.integers(0, 1 << 63, size=distinct, dtype=np.uint64)
    keys = pool[rng.integers(0, distinct, size=count)] if count else np.zeros(0, np.uint64)
    if count > 10:
        keys[: count // 10] &= np.uint64((1 << min(bits, 12)) - 1)  # a crowd in the low digits
    vals = np.arange(count, dtype=np.uint64)
    k, v = host_ctx.debug_sort_pairs(keys, vals, bits)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(k, keys[order])
    assert np.array_equal(v, vals[order])


@pytest.mark.parametrize("directed", [True, False])
def test_hub_groups_match_oracle(ldl, directed):
    """A hub-table budget below any hub's table makes every hub sweep run
    one hub per group (static build and batches): the whole state still
    equals the oracle's."""
    from synth import EdgeStream, csr_from_arcs, rmat_directed, rmat_stream
    g = rmat_directed(scale=14, arcs=1 << (18 if directed else 19), seed=61)
    s, d, w = g.arcs()
    if directed:
        bs = rmat_stream(g, batches=4, size=2000, seed=61)
        deg = np.bincount(s, minlength=g.n) + np.bincount(d, minlength=g.n)
    else:
        g = csr_from_arcs(g.n, s, d, w, directed=False)
        st = EdgeStream.from_graph(g, 61)
        bs = [random_batch(st, 1200, 500, 300, 8, 61 + t) for t in range(4)]
        deg = np.diff(g.row_ptr)
    assert (deg > 2048).sum() >= 8  # hubs above the last bin
    lib = ldl.load()
    lib.ldl_debug_hub_table_slots(1 << 12)
    try:
        o = Oracle(g)
        d = ldl.LDL.from_graph(g)
        msgs = compare_states(o, d, "create")
        assert not msgs, "\n".join(msgs[:8])
        for t, b in enumerate(bs):
            assert o.apply(b) == 0
            d.apply(b)
            msgs = compare_states(o, d, f"batch {t}")
            assert not msgs, "\n".join(msgs[:8])
    finally:
        lib.ldl_debug_hub_table_slots(0)


def test_batch_estimate_covers_observed_growth(ldl):
    """ldl_batch_estimate_bytes learns from the batches it has seen: after a
    batch, the estimate for a batch of the same size covers the device memory
    that batch added."""
    import ctypes

    import torch
    from synth import rmat_directed, rmat_stream
    g = rmat_directed(scale=14, arcs=1 << 18, seed=62)
    bs = rmat_stream(g, batches=2, size=20000, seed=62)
    d = ldl.LDL.from_graph(g)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    d.apply(bs[0])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    est = ctypes.c_int64()
    assert ldl.load().ldl_batch_estimate_bytes(d._h, len(bs[1]), ctypes.byref(est)) == 0
    assert est.value >= free0 - free1 > 0
