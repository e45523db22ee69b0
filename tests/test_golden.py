"""The oracle on the hand-derived fixtures of tests/golden/ (Eq. 1 closed
forms): partition and exact modularity after creation and after each batch."""
import pytest

from oracle import Oracle
from tests.golden_io import blocks_of, cases, load, q_matches


@pytest.mark.parametrize("name", cases())
def test_oracle_reproduces_the_hand_derived_values(name):
    g, batches, expect = load(name)
    o = Oracle(g)
    for t in range(len(expect)):
        if t:
            assert o.apply(batches[t - 1]) == 0
        blocks, q = expect[t]
        assert blocks_of(o.labels()) == blocks
        m, qnum = o.scalars()
        assert q_matches(m, qnum, q), (name, t, m, qnum, q)
