"""Seeded graph and edge-batch generators.

Every random draw comes from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
i-th value of stream (seed, purpose) is mix64(key + (i + 1) * GOLDEN) with
key = mix64(seed * GOLDEN + purpose).  The same (seed, purpose, index) gives
the same value on any machine, so a workload is fully named by its recipe.

Graph shapes stand in for the paper's datasets (its Table III streams, which
are not available here):
  * planted_partition: the SBM-style planted-partition graph of the paper's
    synthetic-recovery study (Sec. IV-E), undirected, int32 weights.
  * rmat_directed: a directed weighted R-MAT graph with the usual skew
    (0.57, 0.19, 0.19, 0.05), standing in for the directed social streams.
  * powerlaw_planted: an LFR-like undirected graph with power-law degrees and
    community sizes and a mixing fraction.
Batches are lists of (src, dst, op, w) int32 quadruples with op in
{INSERT, DELETE, REWEIGHT}; an EdgeStream keeps the current edge set so that
deletes and reweights always name existing edges and inserts name new ones.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

INSERT, DELETE, REWEIGHT = 0, 1, 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_S30, _S27, _S31, _S32, _S11 = (np.uint64(s) for s in (30, 27, 31, 32, 11))


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> _S30)) * _C1
    z = (z ^ (z >> _S27)) * _C2
    return z ^ (z >> _S31)


def splitmix64(seed: int, purpose: int, idx) -> np.ndarray:
    """Value number `idx` (array or scalar) of the stream (seed, purpose), uint64."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([seed], dtype=np.uint64) * _GOLDEN + np.uint64(purpose))
        i = np.asarray(idx, dtype=np.uint64)
        return _mix64(key + (i + np.uint64(1)) * _GOLDEN)


def uniform_u64(seed: int, purpose: int, idx, k) -> np.ndarray:
    """Integers in [0, k) (k < 2**32, scalar or array) from the stream, int64."""
    x = splitmix64(seed, purpose, idx) >> _S32
    with np.errstate(over="ignore"):
        return ((x * np.asarray(k, dtype=np.uint64)) >> _S32).astype(np.int64)


def unit_f64(seed: int, purpose: int, idx) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the stream."""
    return (splitmix64(seed, purpose, idx) >> _S11).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Graph:
    """A weighted graph in CSR form (row_ptr int64[n+1], col int32, w int32).

    Undirected graphs store both arcs of every edge (a symmetric matrix) and
    a self-loop once."""
    n: int
    directed: bool
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    planted: Optional[np.ndarray] = None
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def arcs(self):
        src = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        return src, self.col.astype(np.int64), self.w.astype(np.int64)


def csr_from_arcs(n: int, src, dst, w, directed: bool) -> Graph:
    """CSR of the arc list; duplicate arcs are merged by summing their weights.

    For an undirected graph each (src, dst) edge is mirrored first."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w, dtype=np.int64)
    if not directed:
        off = src != dst
        src, dst, w = (np.concatenate([src, dst[off]]), np.concatenate([dst, src[off]]),
                       np.concatenate([w, w[off]]))
    key = src * n + dst
    order = np.argsort(key, kind="stable")
    key = key[order]
    w = w[order]
    uniq, start = np.unique(key, return_index=True)
    wsum = np.add.reduceat(w, start) if len(key) else w
    s = uniq // n
    d = uniq % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, s + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return Graph(n, directed, row_ptr, d.astype(np.int32), wsum.astype(np.int32))


def planted_partition(n: int = 10000, block: int = 100, intra: int = 5, inter: int = 1,
                      wmax: int = 4, seed: int = 1) -> Graph:
    """Undirected planted partition: n vertices in n/block equal blocks.

    Every vertex draws `intra` partners inside its block and `inter` partners
    in other blocks, so the mean degree is 2*(intra+inter) with a 5:1
    intra/inter ratio at the defaults (about 10 intra and 2 inter neighbours,
    60k edges at n=10,000).  Weights are uniform in 1..wmax; repeated pairs
    sum their weights; there are no self-loops."""
    nb = n // block
    v = np.arange(n, dtype=np.int64)
    srcs, dsts, ws = [], [], []
    for j in range(intra):
        idx = v * (intra + inter) + j
        r = uniform_u64(seed, 11, idx, block - 1)
        loc = v % block
        r = r + (r >= loc)
        srcs.append(v)
        dsts.append((v // block) * block + r)
        ws.append(uniform_u64(seed, 12, idx, wmax) + 1)
    for j in range(inter):
        idx = v * (intra + inter) + intra + j
        ob = uniform_u64(seed, 13, idx, nb - 1)
        ob = ob + (ob >= v // block)
        srcs.append(v)
        dsts.append(ob * block + uniform_u64(seed, 14, idx, block))
        ws.append(uniform_u64(seed, 12, idx, wmax) + 1)
    src = np.concatenate(srcs)
    dst = np.concatenate(dsts)
    w = np.concatenate(ws)
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    g = csr_from_arcs(n, lo, hi, w, directed=False)
    g.planted = (v // block).astype(np.int32)
    g.name = f"planted n={n} blocks={nb}"
    return g


def _rmat_draw(seed: int, purpose: int, base: int, count: int, scale: int, probs):
    """R-MAT endpoints: each recursion level picks a quadrant with
    probabilities (a, b, c, d) quantised to 1/65536; one 64-bit draw serves
    four levels (16 bits each)."""
    a, b, c, _ = probs
    ta, tb, tc = (np.int64(round(x * 65536)) for x in (a, a + b, a + b + c))
    per = (scale + 3) // 4
    idx0 = np.arange(base, base + count, dtype=np.int64)
    src = np.zeros(count, dtype=np.int64)
    dst = np.zeros(count, dtype=np.int64)
    for k in range(per):
        x = splitmix64(seed, purpose, idx0 * per + k)
        for j in range(4):
            if 4 * k + j >= scale:
                break
            u = ((x >> np.uint64(16 * j)) & np.uint64(0xFFFF)).astype(np.int64)
            sb = (u >= tb).astype(np.int64)
            db = (((u >= ta) & (u < tb)) | (u >= tc)).astype(np.int64)
            src = (src << 1) | sb
            dst = (dst << 1) | db
    return src, dst


def rmat_directed(scale: int = 20, arcs: int = 1 << 24, probs=(0.57, 0.19, 0.19, 0.05),
                  wmax: int = 16, seed: int = 2) -> Graph:
    """Directed weighted R-MAT: arcs are drawn until `arcs` distinct non-loop
    arcs have appeared; each keeps the first draw's weight, uniform in 1..wmax."""
    n = 1 << scale
    got_keys = np.zeros(0, dtype=np.int64)
    got_first = np.zeros(0, dtype=np.int64)
    base = 0
    chunk = max(1024, int(arcs * 1.3))
    while True:
        s, d = _rmat_draw(seed, 21, base, chunk, scale, probs)
        keep = s != d
        idx = np.arange(base, base + chunk, dtype=np.int64)[keep]
        key = (s * n + d)[keep]
        allk = np.concatenate([got_keys, key])
        allf = np.concatenate([got_first, idx])
        order = np.argsort(allk, kind="stable")
        allk, allf = allk[order], allf[order]
        u, first = np.unique(allk, return_index=True)
        got_keys, got_first = u, allf[first]
        base += chunk
        if len(got_keys) >= arcs:
            break
        chunk = max(1024, int((arcs - len(got_keys)) * 2))
    sel = np.argsort(got_first, kind="stable")[:arcs]
    key = got_keys[sel]
    w = uniform_u64(seed, 22, got_first[sel], wmax) + 1
    g = csr_from_arcs(n, key // n, key % n, w, directed=True)
    g.name = f"rmat directed scale={scale} arcs={arcs}"
    return g


def cached(name: str, make):
    """Memoise a generated workload on disk (LDL_SYNTH_CACHE, default a
    per-user temp directory) so that tests and the benchmark draw it once per
    machine.  The cache only stores what `make` returns (graph and batches)."""
    import os
    import pickle
    import tempfile
    root = os.environ.get("LDL_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "ldl_synth_cache"))
    os.makedirs(root, exist_ok=True)
    path = os.path.join(root, name + ".pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    obj = make()
    tmp = path + f".{os.getpid()}"
    with open(tmp, "wb") as f:
        pickle.dump(obj, f, protocol=4)
    os.replace(tmp, path)
    return obj


def rmat_workload(nbatches: int, scale: int = 20, arcs: int = 1 << 24, batch: int = 10_000, seed: int = 2,
                  wmax: int = 16):
    """The directed R-MAT stream workload (graph and its first `nbatches`
    batches), cached on disk by recipe."""
    g = cached(f"rmat_graph_s{scale}_a{arcs}_w{wmax}_seed{seed}",
               lambda: rmat_directed(scale=scale, arcs=arcs, wmax=wmax, seed=seed))
    bs = cached(f"rmat_stream_s{scale}_a{arcs}_w{wmax}_seed{seed}_b{batch}_n{nbatches}",
                lambda: rmat_stream(g, batches=nbatches, size=batch, seed=seed, wmax=wmax))
    return g, bs


def multi_graph_workload(graphs: int = 512, nmin: int = 1000, nmax: int = 100_000, steps: int = 8,
                         frac: float = 0.001, seed: int = 4):
    """Many independent graphs for the batched form: vertex counts
    log-uniform in [nmin, nmax]; even graphs directed R-MAT (16 arcs per
    vertex), odd graphs undirected planted partitions
    (100-vertex blocks, weights 1..8); R-MAT graphs have 8 arcs per vertex; every graph gets `steps` batches of
    `frac` of its edges (at least 4 updates), with the planted-partition
    op mix (70% insert, 20% delete, 10% reweight) for odd graphs and 80/20
    insert/delete for the R-MAT ones."""
    u = unit_f64(seed, 111, np.arange(graphs))
    ns = np.exp(np.log(nmin) + u * (np.log(nmax) - np.log(nmin))).astype(np.int64)
    out = []
    for i, n in enumerate(ns.tolist()):
        if i % 2 == 0:
            scale = max(8, int(round(np.log2(n))))
            g = rmat_directed(scale=scale, arcs=8 << scale, wmax=8, seed=seed * 1000 + i)
            size = max(4, int(g.nnz * frac))
            bs = rmat_stream(g, batches=steps, size=size, seed=seed * 1000 + i, wmax=8)
        else:
            nb = max(2, n // 100)
            g = planted_partition(n=nb * 100, block=100, seed=seed * 1000 + i, wmax=8)
            size = max(4, int(g.nnz // 2 * frac))
            bs = planted_stream(g, batches=steps, size=size, seed=seed * 1000 + i, block=100, wmax=8)
        out.append((g, bs))
    return out


def sized_stream(g: Graph, sizes, seed: int, ins_frac: float = 0.8, wmax: int = 16, probs=(0.57, 0.19, 0.19, 0.05)):
    """Batches of the given sizes for an R-MAT graph, drawn as one consistent
    stream (inserts of new R-MAT arcs, deletes of existing arcs)."""
    st = EdgeStream.from_graph(g, seed * 1000 + 13)
    scale = int(g.n).bit_length() - 1

    def sampler(base, cnt):
        return _rmat_draw(seed, 62, base, cnt, scale, probs)
    out = []
    for sz in sizes:
        n_ins = int(round(sz * ins_frac))
        out.append(st.make_batch(n_ins, int(sz) - n_ins, 0, sampler, wmax))
    return out


def random_small_graph(n: int, p: float, directed: bool, wmax: int = 5, seed: int = 0,
                       self_loops: bool = False) -> Graph:
    """Erdos-Renyi style graph for tiny brute-force checks."""
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    if directed:
        keep = (i != j) | self_loops
    else:
        keep = (i < j) | ((i == j) & self_loops)
    i, j = i[keep], j[keep]
    idx = np.arange(len(i))
    sel = unit_f64(seed, 31, idx) < p
    w = uniform_u64(seed, 32, idx, wmax) + 1
    return csr_from_arcs(n, i[sel], j[sel], w[sel], directed)


@dataclass
class EdgeStream:
    """Current edge set of a graph under a stream of batches.

    Keys are src*n+dst for directed graphs and min*n+max for undirected ones;
    weights are kept beside them in key order."""
    n: int
    directed: bool
    keys: np.ndarray
    wts: np.ndarray
    seed: int
    batches_made: int = 0
    draw_counter: int = field(default=0)

    @classmethod
    def from_graph(cls, g: Graph, seed: int) -> "EdgeStream":
        s, d, w = g.arcs()
        if not g.directed:
            keep = s <= d
            s, d, w = s[keep], d[keep], w[keep]
        key = s * g.n + d
        order = np.argsort(key)
        return cls(g.n, g.directed, key[order], w[order], seed)

    def has(self, key: np.ndarray) -> np.ndarray:
        pos = np.searchsorted(self.keys, key)
        pos = np.minimum(pos, len(self.keys) - 1)
        return (len(self.keys) > 0) & (self.keys[pos] == key)

    def canon(self, s: np.ndarray, d: np.ndarray) -> np.ndarray:
        if self.directed:
            return s * self.n + d
        return np.minimum(s, d) * self.n + np.maximum(s, d)

    def make_batch(self, n_ins: int, n_del: int, n_rew: int,
                   sampler: Callable[[int, int], tuple], wmax: int) -> np.ndarray:
        """Draw one batch and apply it to the edge set.

        sampler(base, count) -> (src, dst) proposes insert endpoints from a
        counter window; proposals that are loops, existing edges or repeats
        inside the batch are skipped."""
        t = self.batches_made
        seed = self.seed
        # inserts of new edges
        ins_s, ins_d, ins_k = [], [], []
        need = n_ins
        seen = set()
        tries = 0
        while need > 0 and tries < 64:  # a nearly complete graph may have no new edge left
            tries += 1
            cnt = max(64, 2 * need)
            s, d = sampler(self.draw_counter, cnt)
            self.draw_counter += cnt
            s = np.asarray(s, dtype=np.int64)
            d = np.asarray(d, dtype=np.int64)
            k = self.canon(s, d)
            ok = (s != d) & ~self.has(k)
            for si, di, ki in zip(s[ok], d[ok], k[ok]):
                if need == 0:
                    break
                if ki in seen:
                    continue
                seen.add(int(ki))
                ins_s.append(si)
                ins_d.append(di)
                ins_k.append(ki)
                need -= 1
        ins_w = uniform_u64(seed, 41, np.arange(len(ins_k)) + t * 1_000_003, wmax) + 1
        # deletes and reweights of distinct existing edges
        m = len(self.keys)
        n_old = min(n_del + n_rew, m)
        pick = np.zeros(0, dtype=np.int64)
        if n_old:
            want = 2 * n_old + 64
            if want < m // 4:
                draw = uniform_u64(seed, 42 + t * 7, np.arange(want), m)
                _, first = np.unique(draw, return_index=True)
                pick = draw[np.sort(first)][:n_old]
            if len(pick) < n_old:
                pri = splitmix64(seed, 46 + t * 7, np.arange(m))
                pick = np.argsort(pri, kind="stable")[:n_old]
        dels = pick[:min(n_del, n_old)]
        rews = pick[min(n_del, n_old):]
        rew_w = uniform_u64(seed, 43, np.arange(len(rews)) + t * 1_000_003, wmax) + 1
        flip = uniform_u64(seed, 44, np.arange(len(pick)) + t * 1_000_003, 2)

        def endpoints(idx, fl):
            key = self.keys[idx]
            s, d = key // self.n, key % self.n
            if not self.directed:
                s, d = np.where(fl == 1, d, s), np.where(fl == 1, s, d)
            return s, d
        ds, dd = endpoints(dels, flip[:len(dels)])
        rs, rd = endpoints(rews, flip[len(dels):])
        src = np.concatenate([np.array(ins_s, dtype=np.int64), ds, rs])
        dst = np.concatenate([np.array(ins_d, dtype=np.int64), dd, rd])
        op = np.concatenate([np.full(len(ins_s), INSERT), np.full(len(ds), DELETE),
                             np.full(len(rs), REWEIGHT)]).astype(np.int64)
        w = np.concatenate([ins_w, np.zeros(len(ds), dtype=np.int64), rew_w])
        order = np.argsort(splitmix64(seed, 45 + t * 7, np.arange(len(src))), kind="stable")
        batch = np.stack([src[order], dst[order], op[order], w[order]], axis=1).astype(np.int32)
        # apply to the edge set (keys stay sorted)
        wts = self.wts.copy()
        wts[rews] = rew_w
        keep = np.ones(m, dtype=bool)
        keep[dels] = False
        keys, wts = self.keys[keep], wts[keep]
        ik = np.array(ins_k, dtype=np.int64)
        order = np.argsort(ik, kind="stable")
        ik, iw = ik[order], ins_w[order]
        at = np.searchsorted(keys, ik)
        self.keys, self.wts = np.insert(keys, at, ik), np.insert(wts, at, iw)
        self.batches_made += 1
        return batch


def planted_stream(g: Graph, batches: int = 10, size: int = 100, seed: int = 1,
                   block: int = 100, intra_frac: float = 0.8, wmax: int = 4):
    """Batches for the planted-partition graph: 70% inserts of new edges
    (intra_frac of them inside a block), 20% deletes, 10% reweights."""
    st = EdgeStream.from_graph(g, seed * 1000 + 7)
    n = g.n
    nb = n // block
    n_ins = int(round(size * 0.7))
    n_del = int(round(size * 0.2))
    n_rew = size - n_ins - n_del

    def sampler(base, cnt):
        idx = np.arange(base, base + cnt, dtype=np.int64)
        v = uniform_u64(seed, 51, idx, n)
        intra = unit_f64(seed, 52, idx) < intra_frac
        r = uniform_u64(seed, 53, idx, block - 1)
        r = r + (r >= v % block)
        same = (v // block) * block + r
        ob = uniform_u64(seed, 54, idx, nb - 1)
        ob = ob + (ob >= v // block)
        other = ob * block + uniform_u64(seed, 55, idx, block)
        return v, np.where(intra, same, other)
    return [st.make_batch(n_ins, n_del, n_rew, sampler, wmax) for _ in range(batches)]


def rewire_stream(g: Graph, batches: int = 10, size: int = 500, seed: int = 1, block: int = 100,
                  intra_frac: float = 5.0 / 6.0, wmax: int = 1):
    """Edge rewiring of a planted-partition graph (the dynamic SBM-style
    sequences of the paper's synthetic study): every batch deletes size/2
    existing edges and inserts size/2 new ones drawn by the planted model
    (intra_frac of them inside a block), so the average degree stays put."""
    st = EdgeStream.from_graph(g, seed * 1000 + 17)
    n = g.n
    nb = n // block

    def sampler(base, cnt):
        idx = np.arange(base, base + cnt, dtype=np.int64)
        v = uniform_u64(seed, 56, idx, n)
        intra = unit_f64(seed, 57, idx) < intra_frac
        r = uniform_u64(seed, 58, idx, block - 1)
        r = r + (r >= v % block)
        same = (v // block) * block + r
        ob = uniform_u64(seed, 59, idx, nb - 1)
        ob = ob + (ob >= v // block)
        other = ob * block + uniform_u64(seed, 60, idx, block)
        return v, np.where(intra, same, other)
    half = size // 2
    return [st.make_batch(half, size - half, 0, sampler, wmax) for _ in range(batches)]


def rmat_stream(g: Graph, batches: int = 100, size: int = 10000, seed: int = 2,
                probs=(0.57, 0.19, 0.19, 0.05), wmax: int = 16, ins_frac: float = 0.8):
    """Batches for the directed R-MAT graph: ins_frac inserts of new arcs drawn
    with the same R-MAT skew, the rest deletes of existing arcs."""
    st = EdgeStream.from_graph(g, seed * 1000 + 9)
    scale = int(g.n).bit_length() - 1
    n_ins = int(round(size * ins_frac))
    n_del = size - n_ins

    def sampler(base, cnt):
        return _rmat_draw(seed, 61, base, cnt, scale, probs)
    return [st.make_batch(n_ins, n_del, 0, sampler, wmax) for _ in range(batches)]


def random_batch(st: EdgeStream, n_ins: int, n_del: int, n_rew: int, wmax: int, seed: int):
    """A batch of uniformly random new edges, deletes and reweights (tiny tests)."""
    n = st.n

    def sampler(base, cnt):
        idx = np.arange(base, base + cnt, dtype=np.int64)
        return uniform_u64(seed, 71, idx, n), uniform_u64(seed, 72, idx, n)
    return st.make_batch(n_ins, n_del, n_rew, sampler, wmax)


def config_graph(n: int, degrees: np.ndarray, comm: np.ndarray, mu: float, seed: int) -> Graph:
    """Configuration-model wiring with a mixing fraction: each vertex splits its
    stubs into (1-mu) internal and mu external ones; internal stubs are paired
    at random inside the community, external stubs across the whole graph.
    Loops are dropped and repeated pairs merged (unit weights are summed)."""
    deg = degrees.astype(np.int64)
    ext = np.floor(deg * mu + unit_f64(seed, 81, np.arange(n))).astype(np.int64)
    ext = np.minimum(ext, deg)
    internal = deg - ext
    srcs, dsts = [], []
    # internal stubs, paired inside each community
    stubs = np.repeat(np.arange(n, dtype=np.int64), internal)
    c = comm[stubs].astype(np.int64)
    pri = splitmix64(seed, 82, np.arange(len(stubs)))
    order = np.lexsort((pri, c))
    stubs, c = stubs[order], c[order]
    starts = np.flatnonzero(np.r_[True, c[1:] != c[:-1]])
    seg = np.diff(np.r_[starts, len(c)])
    pos = np.arange(len(c)) - np.repeat(starts, seg)
    even = (pos % 2 == 0) & (pos + 1 < np.repeat(seg, seg))
    srcs.append(stubs[even])
    dsts.append(stubs[np.flatnonzero(even) + 1])
    # external stubs, paired across the graph
    stubs = np.repeat(np.arange(n, dtype=np.int64), ext)
    pri = splitmix64(seed, 83, np.arange(len(stubs)))
    stubs = stubs[np.argsort(pri, kind="stable")]
    h = len(stubs) // 2
    srcs.append(stubs[0:2 * h:2])
    dsts.append(stubs[1:2 * h:2])
    s = np.concatenate(srcs)
    d = np.concatenate(dsts)
    keep = s != d
    s, d = s[keep], d[keep]
    lo, hi = np.minimum(s, d), np.maximum(s, d)
    g = csr_from_arcs(n, lo, hi, np.ones(len(lo), dtype=np.int64), directed=False)
    g.planted = comm.astype(np.int32)
    return g


def powerlaw_planted(n: int = 1 << 24, mean_deg: float = 32.0, deg_exp: float = 2.5,
                     kmax: int = 40000, cmin: int = 50, cmax: int = 50000, comm_exp: float = 1.5,
                     mu: float = 0.2, seed: int = 3) -> Graph:
    """LFR-like undirected graph: Pareto degrees (pdf exponent deg_exp, scaled to
    the requested mean, capped at kmax), power-law community sizes in
    [cmin, cmax] (exponent comm_exp), mixing fraction mu, unit weights."""
    u = unit_f64(seed, 91, np.arange(n))
    a = deg_exp - 1.0
    xmin = mean_deg * (a - 1.0) / a
    deg = np.minimum(np.floor(xmin * (1.0 - u) ** (-1.0 / a)), kmax).astype(np.int64)
    deg = np.maximum(deg, 1)
    # community sizes: inverse-CDF power law on [cmin, cmax]
    sizes = []
    tot = 0
    i = 0
    while tot < n:
        uu = unit_f64(seed, 92, np.arange(i, i + 4096))
        b = 1.0 - comm_exp
        s = np.floor((cmin ** b + uu * (cmax ** b - cmin ** b)) ** (1.0 / b)).astype(np.int64)
        for x in s:
            if tot >= n:
                break
            x = int(min(x, n - tot))
            sizes.append(x)
            tot += x
        i += 4096
    comm = np.repeat(np.arange(len(sizes), dtype=np.int64), sizes)
    perm = np.argsort(splitmix64(seed, 93, np.arange(n)), kind="stable")
    comm = comm[np.argsort(perm, kind="stable")]
    g = config_graph(n, deg, comm, mu, seed)
    g.name = f"powerlaw n={n} mean_deg={mean_deg}"
    return g


def powerlaw_stream(g: Graph, size: int, batches: int, seed: int = 3, ins_frac: float = 0.8,
                    region_factor: int = 4, sizes=None):
    """Batches whose endpoints lie in a seed region: a BFS ball around a seeded
    random vertex grown to at least region_factor*size vertices.  With
    `sizes`, one consistent stream of batches of those sizes instead (the
    region grown for the largest)."""
    n = g.n
    if sizes is not None:
        size = int(max(sizes))
    start = int(uniform_u64(seed, 101, np.array([size]), n)[0])
    want = max(2, region_factor * size)
    seen = np.zeros(n, dtype=bool)
    seen[start] = True
    front = np.array([start], dtype=np.int64)
    region = [front]
    count = 1
    while count < want and len(front):
        nb = np.concatenate([g.col[g.row_ptr[v]:g.row_ptr[v + 1]] for v in front]).astype(np.int64) \
            if len(front) < 4096 else _neighbors(g, front)
        nb = np.unique(nb)
        nb = nb[~seen[nb]]
        seen[nb] = True
        region.append(nb)
        count += len(nb)
        front = nb
    region = np.concatenate(region)
    st = EdgeStream.from_graph(g, seed * 1000 + 11 + size)

    def sampler(base, cnt):
        idx = np.arange(base, base + cnt, dtype=np.int64)
        return (region[uniform_u64(seed, 102, idx, len(region))],
                region[uniform_u64(seed, 103, idx, len(region))])
    out = []
    for sz in (sizes if sizes is not None else [size] * batches):
        n_ins = int(round(sz * ins_frac))
        out.append(_region_batch(st, n_ins, int(sz) - n_ins, sampler, region, seed))
    return out


def _neighbors(g: Graph, vs: np.ndarray) -> np.ndarray:
    starts = g.row_ptr[vs]
    lens = g.row_ptr[vs + 1] - starts
    idx = np.repeat(starts - np.r_[0, np.cumsum(lens)[:-1]], lens) + np.arange(lens.sum())
    return g.col[idx].astype(np.int64)


def _region_batch(st: EdgeStream, n_ins, n_del, sampler, region, seed):
    """Inserts drawn inside the region; deletes of existing edges with an
    endpoint in the region."""
    n = st.n
    inreg = np.zeros(n, dtype=bool)
    inreg[region] = True
    s_all, d_all = st.keys // n, st.keys % n
    cand = np.flatnonzero(inreg[s_all] | inreg[d_all])
    t = st.batches_made
    pri = splitmix64(seed, 104 + t, np.arange(len(cand)))
    k = min(n_del, len(cand))
    pick = cand[np.argsort(pri, kind="stable")[:k]]
    # reuse the generic machinery by temporarily restricting the delete pool
    keys, wts = st.keys, st.wts
    sub = EdgeStream(n, st.directed, keys[pick], wts[pick], st.seed, st.batches_made, st.draw_counter)
    sub.has = st.has  # inserts must be new with respect to the whole graph
    b = sub.make_batch(n_ins, k, 0, sampler, 1)
    st.draw_counter = sub.draw_counter
    # apply to the full edge set
    keep = np.ones(len(keys), dtype=bool)
    keep[pick] = False
    ins = b[b[:, 2] == INSERT]
    ik = st.canon(ins[:, 0].astype(np.int64), ins[:, 1].astype(np.int64))
    allk = np.concatenate([keys[keep], ik])
    allw = np.concatenate([wts[keep], np.ones(len(ik), dtype=np.int64)])
    order = np.argsort(allk, kind="stable")
    st.keys, st.wts = allk[order], allw[order]
    st.batches_made += 1
    return b


# ---------------------------------------------------------------- the largest stream
C5_N = 214_000_000
C5_EDGES = 3_300_000_000
C5_SCALE = 28
_C5_PERM_A = 2_654_435_761  # prime; coprime to 214e6 >> k (= 2^(7-k) * 5^6 * 107)


def c5_size(div_log2: int = 0):
    """(n, distinct undirected edges, R-MAT scale) of the largest stream's
    recipe scaled down by 2^div_log2."""
    return C5_N >> div_log2, C5_EDGES >> div_log2, C5_SCALE - div_log2


def _c5_perm(x: np.ndarray, n: int) -> np.ndarray:
    """Affine id permutation x -> (A x + B) mod n (A coprime to n)."""
    b = int(splitmix64(5, 59, [0])[0]) % n
    return (x % n * (_C5_PERM_A % n) % n + b) % n  # products stay below 2^62 for n < 2^31


def rmat_undirected_c5(div_log2: int = 0, seed: int = 5, chunk: int = 1 << 25,
                       probs=(0.57, 0.19, 0.19, 0.05)) -> Graph:
    """Stand-in for the paper's largest streams (214M vertices, 3.30B edges):
    undirected R-MAT with skew (0.57, 0.19, 0.19, 0.05) at scale 28, draws
    with an id >= 214,000,000 or a loop rejected, distinct edges kept in order
    of first draw until 3.30e9 are reached, an affine id permutation applied,
    unit weights.  div_log2 > 0 scales the recipe down by 2^div_log2 (scale,
    vertex count and edge count alike)."""
    n, target, scale = c5_size(div_log2)
    keys, first = [], []
    base = 0
    have = 0
    while True:
        cnt = min(chunk, int((target - have) * 1.5) + 4096)
        s, d = _rmat_draw(seed, 51, base, cnt, scale, probs)
        ok = (s < n) & (d < n) & (s != d)
        lo, hi = np.minimum(s, d)[ok], np.maximum(s, d)[ok]
        keys.append(lo * n + hi)
        first.append(np.arange(base, base + cnt, dtype=np.int64)[ok])
        base += cnt
        have += int(ok.sum())
        if have < target:
            continue
        allk = np.concatenate(keys)
        allf = np.concatenate(first)
        order = np.argsort(allk, kind="stable")
        allk, allf = allk[order], allf[order]
        u, at = np.unique(allk, return_index=True)
        if len(u) >= target:
            sel = np.argsort(allf[at], kind="stable")[:target]
            key = u[sel]
            break
        keys, first = [u], [allf[at]]
        have = len(u)
    del keys, first
    a = _c5_perm(key // n, n)
    b = _c5_perm(key % n, n)
    del key
    # distinct undirected edges: both arcs of each, sorted by (row, col)
    arc = np.concatenate([a * n + b, b * n + a])
    del a, b
    arc.sort()
    src = arc // n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(src, minlength=n))
    col = (arc % n).astype(np.int32)
    del arc, src
    g = Graph(n, False, row_ptr, col, np.ones(len(col), dtype=np.int32))
    g.name = f"rmat undirected c5 n={n} edges={target}"
    return g


def c5_stream(g: Graph, batches: int, seed: int = 5, max_size: int = 1_000_000, wmax: int = 4,
              probs=(0.57, 0.19, 0.19, 0.05)):
    """Batches of the largest stream: sizes log-uniform in [10, max_size], each
    70% inserts (R-MAT draws with the graph's skew, ids permuted as the
    graph's; an insert of an edge that exists adds its weight), 20% deletes
    and 10% reweights (to 1..wmax) of distinct edges of the initial graph (no
    edge is deleted twice or reweighted after its delete), in a seeded
    shuffled order.  Vectorised: nothing is copied per batch."""
    n = g.n
    scale = max(1, int(n - 1).bit_length())
    u = unit_f64(seed, 81, np.arange(batches))
    sizes = np.floor(10.0 ** (1.0 + u * (np.log10(max_size) - 1.0))).astype(np.int64)
    n_del = np.round(sizes * 0.2).astype(np.int64)
    n_rew = np.round(sizes * 0.1).astype(np.int64)
    n_ins = sizes - n_del - n_rew
    # initial undirected edges (u < v) by index
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    up = src < g.col
    eu, ev = src[up], g.col[up].astype(np.int64)
    del src, up
    m = len(eu)
    need = int(n_del.sum() + n_rew.sum())
    if need > m:
        raise ValueError("stream deletes and reweights more edges than the graph has")
    pick = np.zeros(0, dtype=np.int64)
    want = need + 64
    while len(pick) < need:
        want = 2 * want
        draw = uniform_u64(seed, 82, np.arange(want), m)
        _, at = np.unique(draw, return_index=True)
        pick = draw[np.sort(at)]
    pick = pick[:need]
    out = []
    pos = 0
    ins_base = 0
    for t in range(batches):
        nd, nr, ni = int(n_del[t]), int(n_rew[t]), int(n_ins[t])
        dsel = pick[pos:pos + nd]
        rsel = pick[pos + nd:pos + nd + nr]
        pos += nd + nr
        got_s, got_d = [], []
        have = 0
        while have < ni:
            cnt = 2 * (ni - have) + 64
            s, d = _rmat_draw(seed, 83, ins_base, cnt, scale, probs)
            ins_base += cnt
            ok = (s < n) & (d < n) & (s != d)
            s, d = _c5_perm(s[ok], n), _c5_perm(d[ok], n)
            got_s.append(s[:ni - have])
            got_d.append(d[:ni - have])
            have += len(got_s[-1])
        isrc, idst = np.concatenate(got_s), np.concatenate(got_d)
        iw = uniform_u64(seed, 84, np.arange(ni) + t * 1_000_003, wmax) + 1
        rw = uniform_u64(seed, 85, np.arange(nr) + t * 1_000_003, wmax) + 1
        flip = uniform_u64(seed, 86, np.arange(nd + nr) + t * 1_000_003, 2) == 1
        ds = np.where(flip[:nd], ev[dsel], eu[dsel])
        dd = np.where(flip[:nd], eu[dsel], ev[dsel])
        rs = np.where(flip[nd:], ev[rsel], eu[rsel])
        rd = np.where(flip[nd:], eu[rsel], ev[rsel])
        bsrc = np.concatenate([isrc, ds, rs])
        bdst = np.concatenate([idst, dd, rd])
        op = np.concatenate([np.full(ni, INSERT), np.full(nd, DELETE), np.full(nr, REWEIGHT)])
        w = np.concatenate([iw, np.zeros(nd, dtype=np.int64), rw])
        order = np.argsort(splitmix64(seed, 87 + t * 7, np.arange(len(bsrc))), kind="stable")
        out.append(np.stack([bsrc[order], bdst[order], op[order], w[order]], axis=1).astype(np.int32))
    return out


# ---- the same draws with torch tensors (a GPU builds the largest graphs in
# seconds); bit-identical to the numpy versions above.
def _i64(x: int) -> int:
    """A uint64 constant as the int64 with the same bits."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= 1 << 63 else x


def _lsr_t(z, k: int):
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64_t(z):
    z = (z ^ _lsr_t(z, 30)) * _i64(0xBF58476D1CE4E5B9)
    z = (z ^ _lsr_t(z, 27)) * _i64(0x94D049BB133111EB)
    return z ^ _lsr_t(z, 31)


def splitmix64_t(seed: int, purpose: int, idx):
    """splitmix64 on an int64 torch tensor of indices (values as int64 bits)."""
    key = _i64(int(_mix64(np.array([seed], dtype=np.uint64) * _GOLDEN + np.uint64(purpose))[0]))
    return _mix64_t(key + (idx + 1) * _i64(0x9E3779B97F4A7C15))


def _rmat_draw_t(seed: int, purpose: int, base: int, count: int, scale: int, probs, device):
    import torch
    a, b, c, _ = probs
    ta, tb, tc = (int(round(x * 65536)) for x in (a, a + b, a + b + c))
    per = (scale + 3) // 4
    idx0 = torch.arange(base, base + count, dtype=torch.int64, device=device)
    src = torch.zeros(count, dtype=torch.int64, device=device)
    dst = torch.zeros(count, dtype=torch.int64, device=device)
    for k in range(per):
        x = splitmix64_t(seed, purpose, idx0 * per + k)
        for j in range(4):
            if 4 * k + j >= scale:
                break
            u = _lsr_t(x, 16 * j) & 0xFFFF if j else x & 0xFFFF
            sb = (u >= tb).to(torch.int64)
            db = (((u >= ta) & (u < tb)) | (u >= tc)).to(torch.int64)
            src = (src << 1) | sb
            dst = (dst << 1) | db
    return src, dst


def rmat_undirected_c5_t(div_log2: int = 0, seed: int = 5, device="cuda", chunk: int = 1 << 27,
                         probs=(0.57, 0.19, 0.19, 0.05)) -> Graph:
    """rmat_undirected_c5 built with torch on `device` (same graph, bit for
    bit); the CSR comes back in host memory."""
    import torch
    n, target, scale = c5_size(div_log2)
    keys, first = [], []
    base = 0
    have = 0
    while True:
        cnt = min(chunk, int((target - have) * 1.5) + 4096)
        s, d = _rmat_draw_t(seed, 51, base, cnt, scale, probs, device)
        ok = (s < n) & (d < n) & (s != d)
        lo, hi = torch.minimum(s, d)[ok], torch.maximum(s, d)[ok]
        keys.append(lo * n + hi)
        first.append(torch.arange(base, base + cnt, dtype=torch.int64, device=device)[ok])
        del s, d, ok, lo, hi
        base += cnt
        have += int(keys[-1].numel())
        if have < target:
            continue
        allk = torch.cat(keys)
        allf = torch.cat(first)
        keys, first = [], []
        allk, order = torch.sort(allk, stable=True)
        allf = allf[order]
        del order
        u, cts = torch.unique_consecutive(allk, return_counts=True)
        starts = torch.cumsum(cts, 0) - cts
        f = allf[starts]
        del allk, allf, cts, starts
        if u.numel() >= target:
            sel = torch.sort(f, stable=True).indices[:target]
            key = u[sel]
            del u, f, sel
            break
        keys, first = [u], [f]
        have = int(u.numel())
    b0 = int(splitmix64(5, 59, [0])[0]) % n
    pa = _C5_PERM_A % n
    a_ = ((key // n) % n * pa % n + b0) % n
    b_ = ((key % n) % n * pa % n + b0) % n
    del key
    arc = torch.cat([a_ * n + b_, b_ * n + a_])
    del a_, b_
    arc = torch.sort(arc).values
    src = arc // n
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(torch.bincount(src, minlength=n), 0)
    col = (arc % n).to(torch.int32)
    del arc, src
    g = Graph(n, False, row_ptr.cpu().numpy(), col.cpu().numpy(), np.ones(int(col.numel()), dtype=np.int32))
    del row_ptr, col
    g.name = f"rmat undirected c5 n={n} edges={target}"
    return g
