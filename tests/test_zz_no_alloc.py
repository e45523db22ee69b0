"""The allocation-free copy of changed labels (GB300 only).

Callers that cannot allocate device memory while running use
ldl_copy_changed_noalloc; it must return exactly what ldl_copy_changed
returns.  Checked on two batches in a row, through the C ABI.  This file is
collected last so that a failure here stops a -x run only after every other
test has run.
"""
import numpy as np
import pytest

from synth import rmat_directed, rmat_stream

pytestmark = pytest.mark.gpu


def test_noalloc_copy_matches_copy_changed():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2502_18497_gb300 import LDL
    g = rmat_directed(scale=12, arcs=1 << 16, seed=31)
    d = LDL.from_graph(g)
    seen = 0
    for b in rmat_stream(g, batches=2, size=400, seed=31):
        d.apply(b)
        ids, lab = d.changed()
        ids2, lab2 = d.changed_noalloc()
        assert np.array_equal(ids, ids2)
        assert np.array_equal(lab, lab2)
        assert np.array_equal(lab2, d.labels()[ids2])
        seen += len(ids)
    assert seen > 0
