"""Batched and served execution forms (GB300 only).

Both forms run many independent graphs at once; neither may change any
graph's result.  Each graph is compared bit for bit with its own oracle run
(the result it reaches alone), after batches applied concurrently (batched
form) or submitted interleaved from several producer threads (served form).
"""
import ctypes
import threading

import pytest

from oracle import Oracle
from synth import planted_partition, planted_stream, rmat_directed, rmat_stream
from tests.parity import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


def _graphs(count):
    out = []
    for i in range(count):
        if i % 2 == 0:
            g = rmat_directed(scale=11 + i % 3, arcs=1 << (15 + i % 3), seed=40 + i)
            bs = rmat_stream(g, batches=3, size=300, seed=40 + i)
        else:
            g = planted_partition(n=1500 + 500 * i, block=50, seed=40 + i)
            bs = planted_stream(g, batches=3, size=150, seed=40 + i, block=50, intra_frac=0.5)
        out.append((g, bs))
    return out


def test_batched_form_matches_each_graph_alone(torch_mod):
    from paper_2502_18497_gb300 import LDL, apply_batches
    work = _graphs(6)
    streams = [torch_mod.cuda.Stream() for _ in work]
    gpus = [LDL.from_graph(g, stream=s.cuda_stream) for (g, _), s in zip(work, streams)]
    oracles = [Oracle(g) for g, _ in work]
    for step in range(3):
        apply_batches(gpus, [bs[step] for _, bs in work], threads=4)
        for o, (_, bs) in zip(oracles, work):
            assert o.apply(bs[step]) == 0
    for k, (o, d) in enumerate(zip(oracles, gpus)):
        msgs = compare_states(o, d, f"graph {k}")
        assert not msgs, "\n".join(msgs[:6])


def test_batched_form_full_size(torch_mod):
    """The batched-form workload at its benchmark size: 512 independent graphs
    (vertex counts log-uniform 10^3..10^5, even graphs directed R-MAT, odd
    graphs undirected planted partitions, ~115M stored entries), two steps of
    0.1%-of-edges batches applied to all graphs at once from 16 host threads,
    every graph then compared with its own oracle run (partition, hierarchy
    arrays, community totals and the exact numerator)."""
    from paper_2502_18497_gb300 import LDL, apply_batches
    from synth import multi_graph_workload
    work = multi_graph_workload(512, steps=2)
    streams = [torch_mod.cuda.Stream() for _ in range(16)]
    gpus = [LDL.from_graph(g, stream=streams[k % 16].cuda_stream) for k, (g, _) in enumerate(work)]
    for step in range(2):
        apply_batches(gpus, [bs[step] for _, bs in work], threads=16)
    torch_mod.cuda.synchronize()
    for k, ((g, bs), d) in enumerate(zip(work, gpus)):
        o = Oracle(g)
        for b in bs:
            assert o.apply(b) == 0
        msgs = compare_states(o, d, f"graph {k}", adjacency=(k % 32 == 0))
        assert not msgs, "\n".join(msgs[:6])
        d.close()


def test_served_form_alone_equals_mix(torch_mod):
    from paper_2502_18497_gb300 import Server
    work = _graphs(4)
    srv = Server(workers=3)
    streams = [torch_mod.cuda.Stream() for _ in work]
    gpus = [srv.admit(g, stream=s.cuda_stream) for (g, _), s in zip(work, streams)]
    tickets = {k: [] for k in range(len(work))}
    lock = threading.Lock()

    def producer(ks):
        for step in range(3):
            for k in ks:
                t = srv.submit(gpus[k], work[k][1][step])
                with lock:
                    tickets[k].append(t)

    th = [threading.Thread(target=producer, args=(ks,)) for ks in ([0, 2], [1, 3])]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for k in tickets:
        for t in tickets[k]:
            st, res, queue_us, service_us = srv.wait(t)
            assert st == 0 and service_us > 0 and queue_us >= 0
    for k, ((g, bs), d) in enumerate(zip(work, gpus)):
        o = Oracle(g)
        for b in bs:
            assert o.apply(b) == 0
        msgs = compare_states(o, d, f"tenant {k}")
        assert not msgs, "\n".join(msgs[:6])
    srv.close()


def test_served_form_defers_batches_under_a_memory_cap(torch_mod):
    """Per-batch admission by free memory: with the server told the device
    has almost no free memory, requests that would overlap running ones are
    deferred until those finish (each runs alone when nothing else runs), the
    work still completes, and every tenant's state equals its oracle run."""
    from paper_2502_18497_gb300 import Server
    work = _graphs(4)
    srv = Server(workers=4)
    streams = [torch_mod.cuda.Stream() for _ in work]
    gpus = [srv.admit(g, stream=s.cuda_stream) for (g, _), s in zip(work, streams)]
    srv.debug_free_bytes(1)  # nothing fits beside a running request
    tickets = []
    for step in range(3):
        for k in range(len(work)):
            tickets.append(srv.submit(gpus[k], work[k][1][step]))
    for t in tickets:
        st, res, queue_us, service_us = srv.wait(t)
        assert st == 0 and service_us > 0
    deferred, retried = srv.stats()
    assert deferred > 0
    srv.debug_free_bytes(-1)
    for k, ((g, bs), d) in enumerate(zip(work, gpus)):
        o = Oracle(g)
        for b in bs:
            assert o.apply(b) == 0
        msgs = compare_states(o, d, f"tenant {k}")
        assert not msgs, "\n".join(msgs[:6])
    srv.close()


def test_admission_refuses_what_does_not_fit(torch_mod):
    from paper_2502_18497_gb300 import Server, ldl
    srv = Server(workers=1)
    p = ldl.make_params(directed=True)
    h = ctypes.c_void_p()
    # 2^31-2 vertices with 2^40 arcs cannot fit; nothing is read or allocated
    rc = ldl.load().ldl_server_admit(srv._h, ctypes.byref(p), (1 << 31) - 2, 1 << 40, None, None, None,
                                     ctypes.byref(h))
    assert rc == ldl.LDL_E_NOMEM and not h.value
    srv.close()
