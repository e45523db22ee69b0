"""Checkpoint / resume of the hierarchy and growth of the vertex set through
the C ABI (GB300 only): a context saved with ldl_save and resumed with
ldl_load continues exactly as the saved one and as the oracle; ldl_grow adds
isolated vertices like the oracle's growth, and later batches connecting
them match the oracle bit for bit."""
import os

import numpy as np
import pytest

from oracle import Oracle
from synth import EdgeStream, planted_partition, planted_stream, random_batch, rmat_directed, rmat_stream
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


def _same(o, d, where):
    msgs = compare_states(o, d, where)
    assert not msgs, "\n".join(msgs[:8])


@pytest.mark.parametrize("directed", [False, True])
def test_save_and_load_resume_exactly(ldl, tmp_path, directed):
    if directed:
        g = rmat_directed(scale=12, arcs=1 << 16, seed=51)
        bs = rmat_stream(g, batches=6, size=500, seed=51)
    else:
        g = planted_partition(n=3000, block=50, seed=51)
        bs = planted_stream(g, batches=6, size=120, seed=51, block=50)
    o = Oracle(g, gamma_num=3, gamma_den=2)
    d = ldl.LDL.from_graph(g, gamma_num=3, gamma_den=2)
    for b in bs[:3]:
        assert o.apply(b) == 0
        d.apply(b)
    path = str(tmp_path / "h.ldl")
    d.save(path)
    r = ldl.LDL.load(path)
    assert r.n == g.n and r.directed == directed
    _same(o, r, "loaded")
    for t, b in enumerate(bs[3:]):
        assert o.apply(b) == 0
        d.apply(b)
        r.apply(b)
        _same(o, r, f"loaded, batch {t}")
        _same(o, d, f"original, batch {t}")
    r.close()
    d.close()


def test_load_rejects_bad_files(ldl, tmp_path):
    p = tmp_path / "bad.ldl"
    p.write_bytes(b"not a checkpoint at all")
    with pytest.raises(ldl.LdlError) as e:
        ldl.LDL.load(str(p))
    assert e.value.status == ldl.LDL_E_INVALID
    g = planted_partition(n=500, block=50, seed=52)
    d = ldl.LDL.from_graph(g)
    good = tmp_path / "good.ldl"
    d.save(str(good))
    data = good.read_bytes()
    (tmp_path / "cut.ldl").write_bytes(data[: len(data) // 2])
    with pytest.raises(ldl.LdlError) as e:
        ldl.LDL.load(str(tmp_path / "cut.ldl"))
    assert e.value.status == ldl.LDL_E_INVALID
    with pytest.raises(ldl.LdlError):
        ldl.LDL.load(str(tmp_path / "missing.ldl"))


@pytest.mark.parametrize("directed", [False, True])
def test_growth_matches_the_oracle(ldl, directed):
    if directed:
        g = rmat_directed(scale=11, arcs=1 << 15, seed=53)
        bs = rmat_stream(g, batches=2, size=300, seed=53)
    else:
        g = planted_partition(n=2000, block=50, seed=53)
        bs = planted_stream(g, batches=2, size=100, seed=53, block=50)
    o = Oracle(g)
    d = ldl.LDL.from_graph(g)
    for b in bs:
        assert o.apply(b) == 0
        d.apply(b)
    q0 = d.numerator()
    n2 = g.n + 777
    o.grow(n2)
    d.grow(n2)
    assert d.numerator() == q0
    _same(o, d, "grown")
    # insert-only batches over the grown vertex set (an insert of an edge the
    # earlier batches created adds weight, which is an insert's meaning too)
    st = EdgeStream.from_graph(g, 53)
    st = EdgeStream(n2, st.directed, st.keys // st.n * n2 + st.keys % st.n, st.wts, 53)
    for t in range(4):
        b = random_batch(st, 200, 0, 0, 3, 900 + t)
        assert (b[:, :2] >= g.n).any()
        assert o.apply(b) == 0
        d.apply(b)
        _same(o, d, f"grown, batch {t}")
    d.close()
