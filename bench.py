#!/usr/bin/env python3
"""Throughput of LD-Leiden batch updates on GB300.

Workload: a directed weighted R-MAT graph (a,b,c,d) = (0.57,0.19,0.19,0.05),
2^20 vertices, 2^24 arcs, weights uniform 1..16, built into its initial
hierarchy by the library's static Leiden run, then a stream of batches of
10^4 arc updates (80% inserts of new R-MAT-skewed arcs, 20% deletes of
existing arcs).  A step is one ldl_apply_batch: ingest, statistic repair,
N=2 passes of frontier move / refine / aggregate repair over every level.

Reported (one JSON line on rank 0):
  value      updates/s with the batches already resident in HBM
  e2e        the same through the public API from pinned host buffers, with
             the batch upload and the read-back of the changed labels inside
             the timed region
  roofline   the dominant sweep kernel's algorithmic bytes / its event-timed
             duration, against the measured HBM copy bandwidth
  cpu_baseline  the sequential oracle on the host on a bounded sample
The graph state (adjacency of every level plus per-level arrays) is larger
than the 129 MB L2, so no explicit flush is done between steps.

Multi-GPU (torchrun): every rank runs an independent replica (the path has no
exchange step); value is the total updates of all ranks / the slowest rank.
`--impl reference` times the oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE, ARCS, WMAX, SEED, BATCH = 20, 1 << 24, 16, 2, 10_000
WORKLOAD = ("directed R-MAT (0.57,0.19,0.19,0.05), 2^20 vertices, 2^24 arcs, weights 1..16; "
            "batches of 10^4 arc updates (80% insert / 20% delete)")

# DRAM traffic of the dominant sweep kernel from one ncu capture (dram bytes
# read + written, summed over its launches in one timed step of the default
# workload, divided by the launches that had nodes to sweep: the bins are
# launched unconditionally and an empty launch moves ~23 KB), valid only for
# the sweep source it was taken with (sha256 of csrc/sweep.cu).
NCU_TRAFFIC = {"sha256": "8818a9a99634cdc5b9b9f596981ec682ba71cc56abc199442c4b2f8969263ca9",
               "bytes_per_launch": 45175268, "kernel": "sweep_block128"}


def _set_rmat_scale(scale: int):
    """A smaller R-MAT of the same shape (2^scale vertices, 16 arcs per vertex),
    for profiling captures that must stay small."""
    global SCALE, ARCS, WORKLOAD
    if scale == SCALE:
        return
    SCALE, ARCS = scale, 1 << (scale + 4)
    WORKLOAD = WORKLOAD.replace("2^20 vertices, 2^24 arcs", f"2^{scale} vertices, 2^{scale + 4} arcs")


SWEEP_KERNELS = {"sweep_group8": "k_sweep_group<..., 8>", "sweep_warp": "k_sweep_group<..., 32>",
                 "sweep_block128": "k_sweep_block<..., 128, 2048>", "sweep_block256": "k_sweep_block<..., 256, 4096>",
                 "sweep_cluster": "k_sweep_cluster (8-block cluster, distributed shared-memory hash)",
                 "sweep_hub_acc": "k_hub_acc", "sweep_hub_rest": "hub path set-up + k_hub_eval + k_hub_final"}


def _roofline(ks: dict) -> dict:
    """HBM roofline of the dominant single sweep kernel from the library's
    sweep statistics (algorithmic bytes / event-timed duration); the hub
    path's set-up / evaluation group is several small kernels and is listed
    beside it, not chosen."""
    peak, peak_src = _peaks()
    dom = max((k2 for k2 in ks if k2 != "sweep_hub_rest"), key=lambda k2: ks[k2]["ms"])
    k = ks[dom]
    achieved = k["bytes"] / (k["ms"] / 1e3) / 1e9 if k["ms"] > 0 else 0.0
    return {"bound": "hbm", "kernel": SWEEP_KERNELS.get(dom, dom), "group": dom, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src, "traffic": None,
            "launches": k["launches"], "ms_total": k["ms"],
            "algorithmic_bytes_per_launch": k["bytes"] / max(k["launches"], 1),
            "all_sweep_groups": {n2: {"ms": round(v["ms"], 3), "GB/s": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                                 for n2, v in ks.items()}}


def _workload(nbatches: int):
    from synth import rmat_workload
    return rmat_workload(nbatches, scale=SCALE, arcs=ARCS, batch=BATCH, seed=SEED, wmax=WMAX)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index: int):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(index), "-lms", "50"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, util, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
            try:
                util.append(float(parts[8]))
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
               "reasons": sorted(reasons)}
        if util:
            out["gpu_busy_pct_median"] = statistics.median(util)
        return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(per_rank_updates: int, elapsed: float, device=None):
    """Whole-job throughput over replicas: every rank processed
    `per_rank_updates` in `elapsed` seconds; the job takes as long as its
    slowest rank.  Returns (total updates / max elapsed, max elapsed)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_initialized() else 1
    if ws == 1:
        return per_rank_updates / elapsed, elapsed
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([per_rank_updates], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def oracle_sample(g, batches, warmup: int, steps: int, budget_s: float):
    """The one sampling rule of both CPU measurements (the line's cpu_baseline
    and the reference arm): the oracle as it stands, single-threaded, builds
    its own static Leiden and applies the `warmup` batches the GPU also spends
    on warm-up (both untimed), then times whole batches of the timed region in
    stream order until `steps` batches or `budget_s` seconds are spent.
    Returns (updates/s, batches timed, seconds timed, sample description)."""
    from oracle import Oracle
    t0 = time.perf_counter()
    o = Oracle(g)
    for b in batches[:warmup]:
        assert o.apply(b) == 0
    setup_s = time.perf_counter() - t0
    done, spent, updates = 0, 0.0, 0
    for b in batches[warmup:warmup + steps]:
        t = time.perf_counter()
        assert o.apply(b) == 0
        spent += time.perf_counter() - t
        done += 1
        updates += len(b)
        if spent >= budget_s:
            break
    desc = (f"batches {warmup}..{warmup + done - 1} of the stream ({done} whole batch(es), {updates} updates, "
            f"{spent:.1f} s) after the oracle's own static Leiden and the {warmup} warm-up batch(es) "
            f"({setup_s:.0f} s, untimed); sequential C++, 1 of {os.cpu_count()} cores")
    return updates / spent, done, spent, desc


def cpu_baseline(g, batches, warmup: int, steps: int, budget_s: float):
    ups, _, _, desc = oracle_sample(g, batches, warmup, steps, budget_s)
    return {"value": ups, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": desc}


def run_reference(args):
    """The oracle as the reference arm, on the same workload, metric and
    sampling rule as the GPU line's cpu_baseline (see oracle_sample)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    g, batches = _workload(args.warmup + args.steps)
    ups, done, el, desc = oracle_sample(g, batches, args.warmup, args.steps, args.cpu_budget)
    line = {"metric": "updates/s", "value": ups, "unit": "updates/s", "n_gpus": ws, "steps": done,
            "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "parallelism": "single-threaded oracle"},
            "cpu_baseline": {"value": ups, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": ups, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Batched form: many independent graphs, one batch each per step.
    Reports updates/s of the concurrent multi-stream executor next to the
    plain form (the same contexts updated one after another)."""
    import torch
    from paper_2502_18497_gb300 import LDL, apply_batches
    from synth import cached, multi_graph_workload
    G, W, K = args.graphs, args.warmup, args.steps
    work = cached(f"multi_g{G}_s{W + 2 * K}_seed4_v1", lambda: multi_graph_workload(graphs=G, steps=W + 2 * K))
    streams = [torch.cuda.Stream() for _ in work]
    t0 = time.perf_counter()
    gpus = [LDL.from_graph(g, stream=st.cuda_stream) for (g, _), st in zip(work, streams)]
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    per_step = sum(len(bs[0]) for _, bs in work)
    for s_ in range(W):
        apply_batches(gpus, [bs[s_] for _, bs in work], threads=args.threads)
    torch.cuda.synchronize()
    # plain form: one context after another
    t = time.perf_counter()
    for s_ in range(W, W + K):
        for d, (_, bs) in zip(gpus, work):
            d.apply(bs[s_])
    torch.cuda.synchronize()
    plain = K * per_step / (time.perf_counter() - t)
    # batched form: all contexts concurrently
    lat = []
    t = time.perf_counter()
    for s_ in range(W + K, W + 2 * K):
        t1 = time.perf_counter()
        apply_batches(gpus, [bs[s_] for _, bs in work], threads=args.threads)
        lat.append(time.perf_counter() - t1)
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    ups = K * per_step / el
    line = {"metric": "updates/s", "value": ups, "unit": "updates/s", "n_gpus": 1, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * el / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic", "form": "batched",
            "config": {"workload": f"{G} independent graphs, n log-uniform 1e3..1e5, half directed R-MAT (8 arcs/vertex), "
                                   f"half undirected planted partition; batches of 0.1% of each graph's edges",
                       "edges_total": int(sum(g.nnz if g.directed else g.nnz // 2 for g, _ in work)),
                       "updates_per_step": per_step, "threads": args.threads, "create_s": round(create_s, 1)},
            "plain_value": plain, "speedup_vs_plain": ups / plain,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))}}
    print(json.dumps(line), flush=True)


def run_served(args):
    """Served form: tenants receive batches of log-uniform size (10..10^4) as a
    Poisson stream; the native server runs them with `threads` workers
    (requests of one tenant in order, tenants overlapping).  Reports
    throughput and p50/p99 latency (queue + service) at an arrival rate set to
    `load` x the capacity measured with one worker, next to that one-worker
    (plain) service."""
    import torch
    from paper_2502_18497_gb300 import Server
    from synth import cached, rmat_directed, sized_stream, splitmix64, unit_f64
    T, R = args.tenants, args.requests
    order = (splitmix64(12, 0, np.arange(R)) % np.uint64(T)).astype(int)

    def make():
        out = []
        for k in range(T):
            g = rmat_directed(scale=17, arcs=1 << 21, seed=500 + k)
            cnt = int((order == k).sum()) + 4 * T
            sizes = np.exp(np.log(10) + unit_f64(7, k, np.arange(cnt)) * (np.log(1e4) - np.log(10))).astype(int)
            out.append((g, sized_stream(g, sizes, seed=900 + k)))
        return out
    work = cached(f"served_t{T}_r{R}_v2", make)

    def serve(workers, rate, nreq):
        srv = Server(workers=workers)
        streams = [torch.cuda.Stream() for _ in work]
        gpus = [srv.admit(g, stream=st.cuda_stream) for (g, _), st in zip(work, streams)]
        torch.cuda.synchronize()
        gaps = -np.log(1.0 - unit_f64(11, workers, np.arange(nreq))) / rate if rate else np.zeros(nreq)
        nxt = [0] * T
        tickets, upd = [], 0
        t0 = time.perf_counter()
        due = t0
        for i in range(nreq):
            due += gaps[i]
            while time.perf_counter() < due:
                pass
            k = order[i]
            b = work[k][1][nxt[k]]
            nxt[k] += 1
            tickets.append((time.perf_counter(), srv.submit(gpus[k], b)))
            upd += len(b)
        lat = []
        for ts, tk in tickets:
            st, res, q, sv = srv.wait(tk)
            assert st == 0
            lat.append((q + sv) / 1e3)
        el = time.perf_counter() - t0
        srv.close()
        return upd / el, lat, el
    cap, _, _ = serve(1, 0.0, min(R, 4 * T))            # one worker, back to back: capacity
    # (each serve() call starts from freshly admitted tenants, so the same
    # request sequence is valid again)
    mean_batch = np.mean([len(b) for _, bs in work for b in bs])
    rate = args.load * cap / mean_batch                   # requests per second
    ups1, lat1, _ = serve(1, rate, R)
    upsN, latN, el = serve(args.threads, rate, R)
    line = {"metric": "updates/s", "value": upsN, "unit": "updates/s", "n_gpus": 1, "steps": R, "warmup": 0,
            "ms_per_step": 1e3 * el / R, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic", "form": "served",
            "config": {"workload": f"{T} tenants, each a directed R-MAT 2^17 vertices / 2^21 arcs; batches of "
                                   f"log-uniform 10..10^4 updates arriving as a Poisson stream at "
                                   f"{args.load:.2f} x one-worker capacity", "workers": args.threads,
                       "requests": R},
            "latency_ms": {"p50": float(np.percentile(latN, 50)), "p99": float(np.percentile(latN, 99))},
            "plain": {"updates_per_s": ups1, "latency_ms": {"p50": float(np.percentile(lat1, 50)),
                                                             "p99": float(np.percentile(lat1, 99))}},
            "capacity_one_worker": cap}
    print(json.dumps(line), flush=True)


def run_c5(args):
    """The largest stream's recipe (undirected R-MAT (0.57,0.19,0.19,0.05) at
    scale 28 with ids below 214,000,000, 3.30e9 distinct edges, unit weights;
    batches of log-uniform 10..10^6 updates, 70/20/10 inserts / deletes /
    reweights) scaled down by 2^c5_div so that the hierarchy fits one GPU.
    The graph is drawn on the GPU (bit-identical to the host generator).
    Reports the static build's sweep roofline (frontier = every vertex), the
    plain form (batches back to back from device memory: updates/s, p50/p99
    batch latency) and the served form on the same graph (one worker, batches
    arriving as a Poisson stream at 0.5x and 0.9x the plain capacity: p50/p99
    latency including the wait in the queue)."""
    import torch
    from paper_2502_18497_gb300 import LDL, Server
    from synth import c5_size, c5_stream, unit_f64
    from synth.streams import rmat_undirected_c5_t
    k = args.c5_div
    n, edges, scale = c5_size(k)
    K, W = args.steps, args.warmup
    t0 = time.perf_counter()
    g = rmat_undirected_c5_t(k, device="cuda")
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    bs = c5_stream(g, W + 3 * K, seed=5)
    stream_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    d = LDL.from_graph(g, kernel_stats=1, no_rollback=int(args.no_rollback))
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    static = _roofline(d.kernel_stats())
    d.set_kernel_stats(False)
    free_b, total_b = torch.cuda.mem_get_info()
    print(f"c5: n={n} edges={edges} generate {gen_s:.1f} s, stream {stream_s:.1f} s, create {create_s:.1f} s, "
          f"device memory in use {(total_b - free_b) / 1e9:.1f} of {total_b / 1e9:.1f} GB", file=sys.stderr, flush=True)
    del g
    dev = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    for b in dev[:W]:
        d.apply(b, on_device=True)
        f2, _ = torch.cuda.mem_get_info()
        print(f"c5: warm-up batch of {int(b.shape[0])}: device memory in use {(total_b - f2) / 1e9:.1f} GB",
              file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    # plain form: back to back
    lat, upd = [], 0
    t0 = time.perf_counter()
    for b in dev[W:W + K]:
        t = time.perf_counter()
        d.apply(b, on_device=True)
        lat.append(1e3 * (time.perf_counter() - t))
        upd += int(b.shape[0])
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    cap = upd / plain_s
    mean_batch = float(np.mean([len(b) for b in bs[W:]]))
    served = {}
    srv = Server(workers=1)
    for j, load in enumerate((0.5, 0.9)):
        part = bs[W + (j + 1) * K:W + (j + 2) * K]
        rate = load * cap / mean_batch
        gaps = -np.log(1.0 - unit_f64(13, j, np.arange(len(part)))) / rate
        tickets, u = [], 0
        t0 = time.perf_counter()
        due = t0
        for i, b in enumerate(part):
            due += gaps[i]
            while time.perf_counter() < due:
                pass
            tickets.append(srv.submit(d, b))
            u += len(b)
        sl = []
        for tk in tickets:
            st, _, q, sv = srv.wait(tk)
            assert st == 0, st
            sl.append((q + sv) / 1e3)
        el = time.perf_counter() - t0
        served[str(load)] = {"updates_per_s": u / el, "latency_ms": {"p50": float(np.percentile(sl, 50)),
                                                                      "p99": float(np.percentile(sl, 99))}}
    srv.close()
    line = {"metric": "updates/s", "value": cap, "unit": "updates/s", "n_gpus": 1, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * plain_s / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic", "form": "plain + served (one graph)",
            "config": {"workload": f"undirected R-MAT (0.57,0.19,0.19,0.05) scale {scale}, {n} vertices, {edges} "
                                   f"distinct edges, unit weights (the 214M-vertex / 3.30B-edge recipe / 2^{k}); "
                                   f"batches log-uniform 10..10^6 updates, 70/20/10 insert/delete/reweight",
                       "create_s": round(create_s, 2), "generate_s": round(gen_s, 2), "stream_s": round(stream_s, 2),
                       "atomic_batches": not args.no_rollback, "mean_batch": mean_batch,
                       "device_gb_in_use_after_create": round((total_b - free_b) / 1e9, 1)},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "served": served, "static_build_roofline": static}
    print(json.dumps(line), flush=True)


def run_powerlaw(args):
    """Batch-size sweep on the LFR-like power-law planted partition
    (2^scale vertices, mean degree 32, exponent 2.5, community sizes 50..50,000,
    mixing 0.2): for each batch size B in 10^2..10^6 a fresh instance (same
    initial state) applies `steps` region-localised batches of B updates
    (80% inserts / 20% deletes).  Reports time per batch and updates/s per B,
    and the time ratio per 10x smaller batch."""
    import torch
    from paper_2502_18497_gb300 import LDL
    from synth import cached, powerlaw_planted, powerlaw_stream
    n = 1 << args.scale
    g = cached(f"powerlaw_n{n}_seed3_v1", lambda: powerlaw_planted(n=n, seed=3))
    sizes = [10 ** k for k in range(2, 7) if 10 ** k <= n // 8]
    sweep = {}
    static_roofline, create_s = None, None
    for B in sizes:
        bs = cached(f"powerlaw_n{n}_b{B}_k{args.steps}_seed3_v1",
                    lambda: powerlaw_stream(g, size=B, batches=args.steps, seed=3))
        t0 = time.perf_counter()
        d = LDL.from_graph(g, kernel_stats=1 if static_roofline is None else 0)
        torch.cuda.synchronize()
        if static_roofline is None:  # the static build (frontier = V) of the first instance
            create_s = time.perf_counter() - t0
            static_roofline = _roofline(d.kernel_stats())
            d.set_kernel_stats(False)
        dev = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
        torch.cuda.synchronize()
        times, scanned = [], 0
        for b in dev:
            t = time.perf_counter()
            r = d.apply(b, on_device=True)
            times.append(time.perf_counter() - t)
            scanned += r.edges_scanned
        sweep[B] = {"ms_per_batch": 1e3 * float(np.mean(times)), "updates_per_s": B * len(times) / sum(times),
                    "frontier_entries_per_batch": scanned / len(times)}
        d.close()
    ratios = [sweep[a]["ms_per_batch"] / sweep[b]["ms_per_batch"] for a, b in zip(sizes[1:], sizes[:-1])]
    top = sizes[-1]
    line = {"metric": "updates/s", "value": sweep[top]["updates_per_s"], "unit": "updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": 0, "ms_per_step": sweep[top]["ms_per_batch"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic", "form": "batch-size sweep",
            "config": {"workload": f"power-law planted partition, 2^{args.scale} vertices, {g.nnz // 2} edges, "
                                   f"mean degree 32, mixing 0.2; region-localised batches", "value_at_batch": top},
            "sweep": {str(k): v for k, v in sweep.items()},
            "time_ratio_per_10x_smaller_batch": ratios, "create_s": create_s,
            "static_build_roofline": static_roofline}
    print(json.dumps(line), flush=True)


def run_quality(args):
    """Partition quality beside a static rerun (Sec. IV-A quality metrics,
    Sec. IV-E synthetic recovery): after every batch of the planted-partition
    stream (10,000 vertices, 10 batches of 100) and of the power-law planted
    partition (2^scale vertices, 10 region-localised batches of 1,000), the
    maintained partition is compared with a static Leiden run on the same
    graph snapshot (ldl_create on the level-0 adjacency read back from the
    device): modularity ratio Q_dynamic / Q_static, and ARI / NMI between the
    two partitions and of each against the planted communities.  Quality
    context, not parity: the method is path dependent (Sec. III-H)."""
    import torch
    from paper_2502_18497_gb300 import LDL
    from paper_2502_18497_gb300.quality import ari, nmi
    from synth import planted_partition, planted_stream, powerlaw_planted, powerlaw_stream
    torch.cuda.set_device(0)
    scale = min(args.scale, 22)
    work = [("planted partition 10,000 vertices in 100 blocks, 10 batches of 100", planted_partition(),
             None),
            (f"power-law planted partition 2^{scale} vertices (mean degree 32, mixing 0.2), "
             f"10 region-localised batches of 1,000", powerlaw_planted(n=1 << scale, seed=3), 1000)]
    report = {}
    ratios = []
    for name, g, size in work:
        batches = planted_stream(g) if size is None else powerlaw_stream(g, size=size, batches=10, seed=3)
        d = LDL.from_graph(g)
        rows = []
        for b in batches:
            d.apply(b)
            rp, col, w = d.level_adj(0)
            s = LDL(g.n, rp, col, w.astype(np.int32), directed=g.directed)
            qd, qs = d.modularity(), s.modularity()
            ld, ls = d.labels(), s.labels()
            rows.append({"q_dynamic": qd, "q_static": qs, "ratio": qd / qs if qs else None,
                         "ari_vs_static": ari(ld, ls), "nmi_vs_static": nmi(ld, ls),
                         "ari_vs_planted": ari(ld, g.planted), "nmi_vs_planted": nmi(ld, g.planted),
                         "static_ari_vs_planted": ari(ls, g.planted),
                         "static_nmi_vs_planted": nmi(ls, g.planted)})
            s.close()
            ratios.append(rows[-1]["ratio"])
        d.close()
        mean = {k: float(np.mean([r[k] for r in rows])) for k in rows[0]}
        report[name] = {"per_batch": rows, "mean": mean}
    line = {"metric": "modularity ratio vs a static rerun (and ARI/NMI)", "value": float(np.mean(ratios)),
            "unit": "ratio", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "quality report: " + "; ".join(report)}, "report": report}
    print(json.dumps(line), flush=True)


def run_degree(args):
    """Batch time against average degree (Sec. IV-E, time versus average
    degree as a proxy for the local edge volume the frontier scans): planted
    partitions of 131,000 vertices in 100-vertex blocks with average degree
    2, 4, ..., 64 (5/6 of each vertex's draws inside its block, unit
    weights), each updated by batches of 500 edge changes that rewire the
    graph (250 deletes, 250 inserts drawn by the planted model).  Reports the
    mean device time per batch for every degree and the least-squares slope
    and R^2 of log(time) against log(degree) over degrees >= 8 (the paper fits
    0.57 with its own CPU implementation; the shape, not the constant, is
    what carries over).  ARI against the planted blocks is reported beside it."""
    import torch
    from paper_2502_18497_gb300 import LDL
    from paper_2502_18497_gb300.quality import ari
    from synth import planted_partition, rewire_stream
    torch.cuda.set_device(0)
    n, W, K = 131_000, max(args.warmup, 1), max(args.steps, 5)
    rows = []
    for dbar in (2, 4, 8, 16, 32, 64):
        k = dbar // 2
        intra = max(1, int(round(k * 5 / 6)))
        g = planted_partition(n=n, block=100, intra=intra, inter=k - intra, wmax=1, seed=7 + dbar)
        batches = rewire_stream(g, batches=W + K, size=500, seed=7 + dbar)
        d = LDL.from_graph(g)
        dev = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in batches]
        for b in dev[:W]:
            d.apply(b, on_device=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        scanned = 0
        e0.record()
        for b in dev[W:]:
            scanned += d.apply(b, on_device=True).edges_scanned
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        rows.append({"avg_degree": 2.0 * g.nnz / 2 / n, "nominal_degree": dbar, "ms_per_batch": ms,
                     "updates_per_s": 500 / (ms / 1e3), "edges_scanned_per_batch": scanned / K,
                     "ari_vs_planted": ari(d.labels(), g.planted)})
        d.close()
    fit = [r for r in rows if r["nominal_degree"] >= 8]
    x = np.log([r["avg_degree"] for r in fit])
    y = np.log([r["ms_per_batch"] for r in fit])
    slope, icept = np.polyfit(x, y, 1)
    pred = slope * x + icept
    r2 = 1.0 - float(np.sum((y - pred) ** 2) / np.sum((y - y.mean()) ** 2))
    line = {"metric": "log-log slope of batch time vs average degree (degrees >= 8)", "value": float(slope),
            "unit": "slope", "r2": r2, "higher_is_better": False, "n_gpus": 1, "steps": K, "warmup": W,
            "data": "synthetic", "config": {"workload": "planted partitions 131,000 vertices, 100-vertex blocks, average "
                                            "degree 2..64, batches of 500 rewiring edge changes"},
            "per_degree": rows}
    print(json.dumps(line), flush=True)


def run_autotune(args):
    """Coordinate-descent tuning of the sweep scheduling knobs on the R-MAT
    stream (each candidate re-checked to give the same partition); prints the
    best knobs and every candidate's time per batch."""
    import torch
    from paper_2502_18497_gb300.autotune import tune
    g, batches = _workload(args.steps + 1)
    torch.cuda.synchronize()
    res = tune(g, batches, cache=args.autotune_cache, key=f"rmat{SCALE}_b{BATCH}")
    line = {"metric": "updates/s", "value": BATCH / (res["ms_per_batch"] / 1e3), "unit": "updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": res["ms_per_batch"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic", "form": "autotune",
            "config": {"workload": WORKLOAD}, "best": {"bin_deg": res["bin_deg"],
                                                       "cluster_max_deg": res["cluster_max_deg"]},
            "default_ms_per_batch": res["default_ms_per_batch"], "candidates": res["candidates"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 50 for the R-MAT stream and its reference arm, else 20)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=30.0,
                    help="seconds of timed oracle batches (cpu_baseline and the reference arm)")
    ap.add_argument("--stage-times", action="store_true", help="per-stage device times (adds syncs)")
    ap.add_argument("--no-rollback", action="store_true",
                    help="contexts without the per-batch rollback snapshot and undo log (ldl_params.no_rollback)")
    ap.add_argument("--workload", default="rmat",
                    choices=["rmat", "batched", "served", "powerlaw", "autotune", "quality", "degree", "c5"])
    ap.add_argument("--autotune-cache", default=None, help="autotune: JSON file the result is merged into")
    ap.add_argument("--scale", type=int, default=24, help="powerlaw: log2 of the vertex count")
    ap.add_argument("--graphs", type=int, default=512, help="batched form: number of graphs")
    ap.add_argument("--threads", type=int, default=16, help="batched/served: host worker threads")
    ap.add_argument("--tenants", type=int, default=16, help="served form: graphs")
    ap.add_argument("--requests", type=int, default=400, help="served form: requests")
    ap.add_argument("--rmat-scale", type=int, default=SCALE,
                    help="R-MAT workload: log2 of the vertex count (default: the full-size stream)")
    ap.add_argument("--load", type=float, default=0.9, help="served form: arrival rate / one-worker capacity")
    ap.add_argument("--c5-div", type=int, default=4,
                    help="c5: log2 of the factor the 214M-vertex / 3.30B-edge recipe is scaled down by")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 50 if args.workload == "rmat" else 20
    _set_rmat_scale(args.rmat_scale)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "powerlaw":
        return run_powerlaw(args)
    if args.workload == "autotune":
        return run_autotune(args)
    if args.workload == "quality":
        return run_quality(args)
    if args.workload == "degree":
        return run_degree(args)
    if args.workload == "c5":
        return run_c5(args)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2502_18497_gb300 import LDL, ldl as binding

    W, K = args.warmup, args.steps
    g, batches = _workload(W + 2 * K)
    t0 = time.perf_counter()
    d = LDL.from_graph(g, kernel_stats=1, no_rollback=int(args.no_rollback))
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    # the static build sweeps every vertex first (frontier = V): the sweeps'
    # roofline when the frontier fills the GPU
    static_roofline = _roofline(d.kernel_stats())
    dev = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in batches[:W + K]]
    for b in dev[:W]:
        d.apply(b, on_device=True)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    d.set_kernel_stats(True)
    if args.stage_times:
        d.set_timing(True)
    clocks = ClockSampler(local)
    launches0 = binding.launch_count()
    scanned = 0
    work = {}
    lat = []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record()
    for b in dev[W:W + K]:
        t = time.perf_counter()
        r = d.apply(b, on_device=True)
        lat.append(time.perf_counter() - t)
        scanned += r.edges_scanned
        for k2, v2 in d.result_dict().items():
            if isinstance(v2, int):
                work[k2] = work.get(k2, 0) + v2
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    ups, el = reduce_over_ranks(K * BATCH, ms / 1e3, device="cuda")
    ms = el * 1e3
    launches = binding.launch_count() - launches0
    clk = clocks.stop()
    ks = d.kernel_stats()
    stage = d.stage_times() if args.stage_times else None
    d.set_kernel_stats(False)
    d.set_timing(False)

    # ---- end to end through the public API from pinned host memory
    host = [torch.from_numpy(np.ascontiguousarray(b)).pin_memory() for b in batches[W + K:W + 2 * K]]
    h2d = d2h = 0
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for b in host:
        d.apply(b)
        ids, labs = d.changed()
        h2d += b.numel() * 4
        d2h += ids.nbytes + labs.nbytes
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t
    e2e_ups, e2e_s = reduce_over_ranks(K * BATCH, e2e_s, device="cuda")
    e2e = {"value": e2e_ups, "unit": "updates/s", "h2d_bytes_per_step": h2d // K,
           "d2h_bytes_per_step": d2h // K}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant sweep kernel
    sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2502_18497_gb300", "csrc", "sweep.cu"), "rb").read()).hexdigest()
    roofline = _roofline(ks)
    if (NCU_TRAFFIC["sha256"] == sha and NCU_TRAFFIC["kernel"] == roofline["group"] and SCALE == 20):
        roofline["traffic"] = NCU_TRAFFIC["bytes_per_launch"]

    line = {"metric": "updates/s", "value": ups, "unit": "updates/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "state larger than L2 (no flush)",
                       "parallelism": "replicas" if ws > 1 else "single GPU", "create_s": round(create_s, 2),
                       "atomic_batches": not args.no_rollback},
            "frontier_edges_per_s": scanned / (ms / 1e3) * ws,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
            "roofline": roofline, "static_build_roofline": static_roofline, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk}
    if stage:
        line["stage_ms_per_step"] = {k2: v / K for k2, v in stage.items()}
        line["work_per_step"] = {k2: v / K for k2, v in work.items()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, batches, W, K, args.cpu_budget)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
