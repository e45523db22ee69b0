"""GPU parity: the CUDA library against the oracle, bit for bit (GB300 only).

Every test builds the same seeded graph and batches for both sides, runs the
oracle on the CPU and the library through its C ABI, and compares the whole
state (hierarchy, labels, strengths, adjacency of every level, community
totals, m and the Eq. 1 numerator) after creation and after every batch.
Integer state must match exactly; the reported modularity within 1e-12
relative.
"""
import os

import numpy as np
import pytest

from oracle import Oracle
from synth import (EdgeStream, planted_partition, planted_stream, random_batch, random_small_graph,
                   rmat_directed, rmat_stream)
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


def _pair(ldl, g, **params):
    o = Oracle(g, **params)
    d = ldl.LDL.from_graph(g, **params)
    return o, d


def _assert_same(o, d, where, **kw):
    msgs = compare_states(o, d, where, **kw)
    assert not msgs, "\n".join(msgs[:12])


@pytest.mark.parametrize("directed", [False, True])
@pytest.mark.parametrize("L,Mst", [(0, 1), (0, 3), (0, 20), (1, 1), (1, 20), (4, 20)])
def test_static_build_small(ldl, directed, L, Mst):
    for seed in range(6):
        g = random_small_graph(12 + 5 * seed, 0.25, directed, wmax=5, seed=seed, self_loops=seed % 2 == 0)
        if not g.nnz:
            continue
        o, d = _pair(ldl, g, L=L, M_static=Mst)
        _assert_same(o, d, f"seed {seed} create")


@pytest.mark.parametrize("directed", [False, True])
def test_random_streams(ldl, directed):
    for seed in range(8):
        g = random_small_graph(20 + 7 * seed, 0.2, directed, wmax=4, seed=50 + seed)
        if not g.nnz:
            continue
        params = dict(L=1 + seed % 4, M_static=2 + seed % 5, M=1 + seed % 5, N=1 + seed % 3)
        o, d = _pair(ldl, g, **params)
        _assert_same(o, d, f"seed {seed} create")
        st = EdgeStream.from_graph(g, seed)
        for t in range(8):
            m = len(st.keys)
            b = random_batch(st, 4, min(3, m), min(2, max(0, m - 3)), 4, seed * 97 + t)
            assert o.apply(b) == 0
            d.apply(b)
            _assert_same(o, d, f"seed {seed} batch {t}")


def test_planted_partition_full(ldl):
    """The 10,000-vertex planted-partition stream: static Leiden, then 10
    batches of 100 updates (70 inserts, 20 deletes, 10 reweights)."""
    g = planted_partition()
    o, d = _pair(ldl, g)
    _assert_same(o, d, "create")
    for t, b in enumerate(planted_stream(g)):
        assert o.apply(b) == 0
        d.apply(b)
        _assert_same(o, d, f"batch {t}")
        assert np.array_equal(o.labels(), np.asarray(d.labels()))


@pytest.mark.parametrize("cluster_max_deg,bin_deg", [(0, None), (32768, None), (0, (16, 64, 256, 1024))])
def test_rmat_directed_reduced(ldl, cluster_max_deg, bin_deg):
    """Directed R-MAT with the paper-stream skew at 2^14 vertices / 2^18 arcs,
    20 batches of 1,000 arc updates (80% inserts, 20% deletes); rows above
    2048 entries swept by the whole-GPU hub path or by block clusters, and
    non-default degree bins (scheduling only: the result must not change)."""
    g = rmat_directed(scale=14, arcs=1 << 18, seed=12)
    o = Oracle(g)
    d = ldl.LDL.from_graph(g, cluster_max_deg=cluster_max_deg, bin_deg=bin_deg)
    _assert_same(o, d, "create", adjacency=False)
    d.set_kernel_stats(True)
    for t, b in enumerate(rmat_stream(g, batches=20, size=1000, seed=12)):
        assert o.apply(b) == 0
        d.apply(b)
        _assert_same(o, d, f"batch {t}", adjacency=(t % 5 == 4))
    ks = d.kernel_stats()
    assert (ks["sweep_cluster"]["launches"] > 0) == (cluster_max_deg > 0)
    assert ks["sweep_hub_acc"]["launches"] > 0 or cluster_max_deg > 0


def test_rmat_directed_full_size(ldl):
    """The benchmark workload at full size (directed R-MAT, 2^20 vertices,
    2^24 arcs): the static build and the first 12 batches of 10^4 updates,
    compared bit for bit after every batch (every level's adjacency after
    the first two, the last and every fourth)."""
    from synth import rmat_workload
    g, bs = rmat_workload(12)
    o, d = _pair(ldl, g)
    _assert_same(o, d, "create")
    for t, b in enumerate(bs):
        assert o.apply(b) == 0
        d.apply(b)
        _assert_same(o, d, f"batch {t}", adjacency=(t < 2 or t % 4 == 3 or t == len(bs) - 1))


@pytest.mark.parametrize("bad,status", [
    ([[0, 10_000, 0, 1]], 2), ([[0, 1, 7, 1]], 1), ([[0, 1, 0, 0]], 1), ([[0, 1, 2, -3]], 4),
    ([[2, 999, 1, 0]], 3), ([[5, 6, 0, 2**31 - 1], [5, 6, 0, 2**31 - 1]], 8),
])
def test_invalid_batches(ldl, bad, status):
    g = planted_partition(n=1000, block=50, seed=7)
    o, d = _pair(ldl, g)
    batch = np.array([[1, 2, 0, 1]] + bad, np.int32)
    assert o.apply(batch) == status
    assert d.try_apply(batch) == status
    _assert_same(o, d, "after rejected batch")


def test_empty_and_null_batches(ldl):
    g = planted_partition(n=1000, block=50, seed=6)
    o, d = _pair(ldl, g)
    s, t, w = int(g.arcs()[0][0]), int(g.arcs()[1][0]), int(g.w[0])
    for b in (np.zeros((0, 4), np.int32), np.array([[s, t, 2, w + 1], [s, t, 2, w]], np.int32)):
        assert o.apply(b) == 0
        d.apply(b)
        _assert_same(o, d, "after null batch")


@pytest.mark.parametrize("size", [100, 1000])
def test_powerlaw_planted_reduced(ldl, size):
    """The LFR-like power-law planted partition at 2^16 vertices (mean degree
    ~28, mixing 0.2), two region-localised batches per batch size, each size
    starting from the same initial state."""
    from synth import powerlaw_planted, powerlaw_stream
    g = powerlaw_planted(n=1 << 16, seed=3)
    o, d = _pair(ldl, g)
    for t, b in enumerate(powerlaw_stream(g, size=size, batches=2, seed=3)):
        assert o.apply(b) == 0
        d.apply(b)
        _assert_same(o, d, f"size {size} batch {t}")


def test_injected_allocation_failure_at_create(ldl):
    """A failing device allocation during ldl_create returns NOMEM and leaves
    nothing behind; the next create succeeds."""
    g = planted_partition(n=1000, block=50, seed=9)
    for k in (1, 5, 40):
        ldl.load().ldl_debug_fail_alloc_after(k)
        with pytest.raises(ldl.LdlError) as e:
            ldl.LDL.from_graph(g)
        assert e.value.status == ldl.LDL_E_NOMEM
    ldl.load().ldl_debug_fail_alloc_after(0)
    o, d = _pair(ldl, g)
    _assert_same(o, d, "after injected failures")


@pytest.mark.parametrize("directed", [False, True])
def test_injected_allocation_failures_during_a_batch_roll_back(ldl, directed):
    """A device allocation that fails in the middle of ldl_apply_batch (after
    the batch began changing the state) returns NOMEM and leaves the whole
    state bit-identical to the oracle's state before the batch; the same batch
    then applies and matches the oracle after it.  Failures are injected at
    the 1st, 2nd, ... allocation of successive attempts until one succeeds."""
    if directed:
        g = rmat_directed(scale=11, arcs=1 << 14, seed=33)
        batches = rmat_stream(g, batches=4, size=3000, seed=33)
    else:
        g = planted_partition(n=2000, block=50, seed=31)
        batches = planted_stream(g, batches=4, size=600, seed=31, block=50)
    o, d = _pair(ldl, g)
    mid_batch = 0
    for t, b in enumerate(batches):
        for k in range(1, 400):
            _, before = ldl.alloc_counts()
            ldl.load().ldl_debug_fail_alloc_after(k)
            st = d.try_apply(b)
            ldl.load().ldl_debug_fail_alloc_after(0)
            if st == 0:
                break
            assert st == ldl.LDL_E_NOMEM, st
            _, after = ldl.alloc_counts()
            mid_batch += after > before
            _assert_same(o, d, f"batch {t} after a failure at allocation {k}")
        else:
            raise AssertionError("the batch never succeeded")
        assert o.apply(b) == 0
        _assert_same(o, d, f"batch {t} applied")
    assert mid_batch > 0


def test_bounded_scan_wait_reports_timeout(ldl):
    """A device scan whose first tile never publishes: the waiting tile gives
    up after its bounded number of polls and the library reports TIMEOUT
    (no hang, and the context-free check leaves the device usable)."""
    assert ldl.load().ldl_debug_scan_wait_timeout() == ldl.LDL_E_TIMEOUT
    g = planted_partition(n=1000, block=50, seed=8)
    o, d = _pair(ldl, g)
    _assert_same(o, d, "create after the timeout check")


def test_hand_derived_fixtures(ldl):
    """The CUDA path on the hand-derived fixtures of tests/golden/: partition
    and exact Eq. 1 numerator after creation and after each batch."""
    from tests.golden_io import blocks_of, cases, load, q_matches
    for name in cases():
        g, batches, expect = load(name)
        d = ldl.LDL.from_graph(g)
        for t in range(len(expect)):
            if t:
                d.apply(batches[t - 1])
            blocks, q = expect[t]
            assert blocks_of(d.labels()) == blocks, name
            m, qnum = d.numerator()
            assert q_matches(m, qnum, q), (name, t, m, qnum, q)


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("LDL_FULL_PARITY") != "1",
                    reason="full-size power-law parity takes tens of minutes (generator and oracle); "
                           "set LDL_FULL_PARITY=1")
def test_powerlaw_planted_full_size(ldl):
    """The power-law planted partition at its benchmark size (2^24 vertices,
    ~242M edges): the static build, then one region-localised stream of
    batches of 10^2, 10^2, 10^3, 10^3, 10^4 and 10^4 updates, compared bit for
    bit after every batch (every level's adjacency after the last)."""
    from synth import powerlaw_planted, powerlaw_stream
    g = powerlaw_planted(n=1 << 24, seed=3)
    sizes = [100, 100, 1000, 1000, 10000, 10000]
    bs = powerlaw_stream(g, size=max(sizes), batches=len(sizes), seed=3, sizes=sizes)
    o, d = _pair(ldl, g)
    _assert_same(o, d, "create", adjacency=False)
    for t, b in enumerate(bs):
        assert o.apply(b) == 0
        d.apply(b)
        _assert_same(o, d, f"batch {t} ({len(b)} updates)", adjacency=(t == len(bs) - 1))
