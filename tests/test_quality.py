"""The partition-quality figures used by the benchmark's quality report (ARI
and NMI, Sec. IV-A / IV-E) against hand-derived values in
tests/golden/quality/ (CPU only), plus the properties that hold at any size."""
import math
import os
import re
from fractions import Fraction

import numpy as np

from paper_2502_18497_gb300.quality import ari, nmi

FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "quality", "ari_nmi.txt")


def _value(expr: str) -> float:
    """A fixture value: a fraction, or a product/quotient of fractions and ln(k)."""
    expr = expr.strip()
    if not re.fullmatch(r"[-0-9/ *()ln.]+", expr):
        raise ValueError(expr)
    if re.fullmatch(r"-?\d+(/\d+)?", expr):
        return float(Fraction(expr))
    tokens = re.findall(r"ln\(\d+\)|\d+|[*/]", expr)
    val, op = None, "*"
    for t in tokens:
        if t in "*/":
            op = t
            continue
        x = math.log(int(t[3:-1])) if t.startswith("ln") else float(t)
        val = x if val is None else (val * x if op == "*" else val / x)
    return val


def _cases():
    out, cur = [], None
    for raw in open(FIXTURE):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tag, _, rest = line.partition(" ")
        if tag == "case":
            cur = {"name": rest}
            out.append(cur)
        elif tag in ("a", "b"):
            cur[tag] = np.array([int(x) for x in rest.split()])
        else:
            cur[tag] = _value(rest)
    return out


def test_fixture_values():
    cases = _cases()
    assert len(cases) == 4
    for c in cases:
        assert abs(ari(c["a"], c["b"]) - c["ari"]) < 1e-12, c["name"]
        assert abs(nmi(c["a"], c["b"]) - c["nmi"]) < 1e-12, c["name"]


def test_symmetry_and_relabelling_invariance():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a = rng.integers(0, 7, 200)
        b = rng.integers(0, 4, 200)
        perm = rng.permutation(7)
        assert abs(ari(a, b) - ari(b, a)) < 1e-12
        assert abs(nmi(a, b) - nmi(b, a)) < 1e-12
        assert abs(ari(perm[a], b) - ari(a, b)) < 1e-12
        assert abs(nmi(perm[a], b) - nmi(a, b)) < 1e-12
        assert -1.0 <= ari(a, b) <= 1.0 and 0.0 <= nmi(a, b) <= 1.0 + 1e-12
        assert abs(ari(a, a) - 1.0) < 1e-12 and abs(nmi(a, a) - 1.0) < 1e-12
