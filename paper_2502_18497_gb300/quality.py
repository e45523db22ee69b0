"""Partition-quality figures for reporting (not on the update path).

The paper compares the partitions its method maintains with those of other
systems by modularity ratio and, on synthetic streams with planted
communities, by the adjusted Rand index (ARI) and normalised mutual
information (NMI) against the planted labels (Sec. IV-A quality metrics,
Sec. IV-E synthetic recovery).  These helpers compute the same figures for
two labelings given as integer arrays, from their contingency table:

  ARI = (sum_ij C(n_ij,2) - E) / ((sum_i C(a_i,2) + sum_j C(b_j,2))/2 - E),
        E = sum_i C(a_i,2) * sum_j C(b_j,2) / C(n,2)
  NMI = 2 I(A;B) / (H(A) + H(B))   (natural logarithms; 1 when both
        labelings are a single cluster)

They run on the host with numpy over label arrays copied from the device and
are used by the benchmark's quality report only.
"""
from __future__ import annotations

import numpy as np


def _contingency(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    if a.shape != b.shape:
        raise ValueError("labelings differ in length")
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    nb = int(bi.max()) + 1 if len(bi) else 1
    pair = ai.astype(np.int64) * nb + bi
    _, nij = np.unique(pair, return_counts=True)
    ni = np.bincount(ai)
    nj = np.bincount(bi)
    return nij.astype(np.float64), ni.astype(np.float64), nj.astype(np.float64), float(len(a))


def ari(a, b) -> float:
    """Adjusted Rand index of two labelings of the same items."""
    nij, ni, nj, n = _contingency(a, b)

    def c2(x):
        return x * (x - 1.0) / 2.0
    s = float(c2(nij).sum())
    sa = float(c2(ni).sum())
    sb = float(c2(nj).sum())
    tot = c2(n)
    if tot == 0:
        return 1.0
    exp = sa * sb / tot
    mx = (sa + sb) / 2.0
    return 1.0 if mx == exp else (s - exp) / (mx - exp)


def nmi(a, b) -> float:
    """Normalised mutual information 2 I / (H_a + H_b) of two labelings."""
    nij, ni, nj, n = _contingency(a, b)
    if n == 0:
        return 1.0
    pa, pb = ni / n, nj / n
    ha = -float(np.sum(pa * np.log(pa)))
    hb = -float(np.sum(pb * np.log(pb)))
    if ha + hb == 0.0:
        return 1.0
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    pair = ai.astype(np.int64) * len(nj) + bi
    keys, cnt = np.unique(pair, return_counts=True)
    pij = cnt / n
    i_idx, j_idx = keys // len(nj), keys % len(nj)
    mi = float(np.sum(pij * np.log(pij / (pa[i_idx] * pb[j_idx]))))
    return max(0.0, 2.0 * mi / (ha + hb))
