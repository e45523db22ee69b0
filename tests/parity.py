"""Helpers that compare the CUDA library's state with the oracle's (tests only)."""
from __future__ import annotations

import numpy as np


def first_diff(a, b):
    d = np.flatnonzero(np.asarray(a) != np.asarray(b))
    return int(d[0]) if len(d) else -1


def compare_states(o, g, where="", adjacency=True, levels=True):
    """Bit-exact comparison of the oracle `o` and the GPU instance `g`.

    Compares the hierarchy height, every per-level node array on alive nodes,
    every level's adjacency, the community totals, m and the Eq. 1 numerator,
    and the reported modularity within 1e-12 relative.  Returns a list of
    mismatch messages (empty when identical)."""
    msgs = []
    if o.top != g.top:
        return [f"{where}: top level oracle={o.top} gpu={g.top}"]
    mo, qo = o.scalars()
    mg, qg = g.numerator()
    if mo != mg:
        msgs.append(f"{where}: m oracle={mo} gpu={mg}")
    if qo != qg:
        msgs.append(f"{where}: Qnum oracle={qo} gpu={qg}")
    ko, ki, e = o.comm()
    kg, kig, eg = g.comm()
    for name, a, b in (("Kout", ko, kg), ("Kin", ki, kig), ("e", e, eg)):
        i = first_diff(a, b)
        if i >= 0:
            msgs.append(f"{where}: {name}[{i}] oracle={a[i]} gpu={b[i]}")
    if levels:
        for r in range(o.top + 1):
            lo_, lg = o.level(r), g.level(r)
            i = first_diff(lo_.alive, lg.alive)
            if i >= 0:
                msgs.append(f"{where}: level {r} alive[{i}] oracle={lo_.alive[i]} gpu={lg.alive[i]}")
                continue
            al = lo_.alive.astype(bool)
            for name in ("lab", "par", "kout", "kin", "cnt"):
                a = getattr(lo_, name)[al]
                b = getattr(lg, name)[al]
                i = first_diff(a, b)
                if i >= 0:
                    v = np.flatnonzero(al)[i]
                    msgs.append(f"{where}: level {r} {name}[{v}] oracle={a[i]} gpu={b[i]}")
            if adjacency:
                ro, co, wo = o.level_adj(r)
                rg, cg, wg = g.level_adj(r)
                if not (np.array_equal(ro, rg) and np.array_equal(co, cg) and np.array_equal(wo, wg)):
                    i = first_diff(ro, rg) if len(ro) == len(rg) else -2
                    msgs.append(f"{where}: level {r} adjacency differs (first row {i}, nnz {len(co)} vs {len(cg)})")
    if mo:
        qf = o.modularity()
        qgf = g.modularity()
        if abs(qf - qgf) > 1e-12 * max(abs(qf), 1e-3):
            msgs.append(f"{where}: modularity {qf} vs {qgf}")
    return msgs
