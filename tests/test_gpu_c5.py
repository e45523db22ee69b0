"""The largest stream's recipe on the GPU (GB300 only): the graph drawn with
torch on the device equals the host generator's bit for bit, and a reduced
replica (scale 17: 104,492 vertices, 1.61M distinct edges, unit weights,
R-MAT hubs) stays bit-identical to the oracle through its static build and
a stream of log-uniform batches with inserts, deletes and reweights."""
import pytest

from oracle import Oracle
from synth import c5_stream, rmat_undirected_c5
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


def test_device_builder_matches_host(ldl):
    import numpy as np
    from synth.streams import rmat_undirected_c5_t
    g = rmat_undirected_c5(11)
    h = rmat_undirected_c5_t(11, device="cuda")
    assert np.array_equal(g.row_ptr, h.row_ptr) and np.array_equal(g.col, h.col)


def test_reduced_replica_matches_oracle(ldl):
    g = rmat_undirected_c5(11)
    bs = c5_stream(g, 6, max_size=20_000)
    o = Oracle(g)
    d = ldl.LDL.from_graph(g)
    msgs = compare_states(o, d, "create")
    assert not msgs, "\n".join(msgs[:8])
    for t, b in enumerate(bs):
        assert o.apply(b) == 0
        d.apply(b)
        msgs = compare_states(o, d, f"batch {t} ({len(b)} updates)")
        assert not msgs, "\n".join(msgs[:8])
