"""Reader of the hand-derived fixtures in tests/golden/ (graph, batches and
the expected partition and exact modularity after creation and each batch)."""
import os

import numpy as np

from synth import DELETE, INSERT, REWEIGHT, csr_from_arcs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
OPS = {"insert": INSERT, "delete": DELETE, "reweight": REWEIGHT}


def cases():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


def load(name):
    """Returns (graph, [batch, ...], [(blocks, (num, den)), ...]); the first
    expectation is after creation, then one per batch."""
    src, dst, w, batches, expect = [], [], [], [], []
    n = directed = None
    cur = None
    blocks = q = None
    for raw in open(os.path.join(GOLDEN, name)):
        line = raw.split("#", 1)[0].split()
        if not line:
            continue
        tag = line[0]
        if tag == "graph":
            directed, n = line[1] == "directed", int(line[2])
        elif tag == "edge":
            src.append(int(line[1]))
            dst.append(int(line[2]))
            w.append(int(line[3]))
        elif tag == "batch":
            cur = []
            batches.append(cur)
        elif tag == "update":
            cur.append([int(line[1]), int(line[2]), OPS[line[3]], int(line[4])])
        elif tag == "expect" and line[1] == "blocks":
            blocks = sorted(tuple(int(x) for x in b.split(",")) for b in line[2:])
        elif tag == "expect" and line[1] == "q":
            q = (int(line[2]), int(line[3]))
            expect.append((blocks, q))
    g = csr_from_arcs(n, src, dst, w, directed)
    return g, [np.array(b, np.int32) for b in batches], expect


def blocks_of(labels):
    groups = {}
    for v, c in enumerate(np.asarray(labels).tolist()):
        groups.setdefault(c, []).append(v)
    return sorted(tuple(sorted(b)) for b in groups.values())


def q_matches(m, qnum, q, gamma_den=1):
    """Q = qnum / (gamma_den * m^2) equals num / den exactly."""
    num, den = q
    return qnum * den == num * gamma_den * m * m
