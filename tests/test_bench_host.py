"""Host-side logic of bench.py (no GPU): the roofline's choice of kernel and
its arithmetic, and the per-launch traffic guard."""
import bench


def _ks(**ms):
    return {k: {"launches": 10.0, "ms": v, "bytes": 1e9 * v, "entries": 1.0} for k, v in ms.items()}


def test_roofline_takes_the_dominant_single_kernel():
    ks = _ks(sweep_group8=1.0, sweep_warp=2.0, sweep_block128=3.0, sweep_block256=0.5, sweep_cluster=0.0,
             sweep_hub_acc=2.5, sweep_hub_rest=9.0)
    r = bench._roofline(ks)
    # the hub path's set-up / evaluation group is several kernels: never chosen
    assert r["group"] == "sweep_block128"
    assert r["kernel"] == bench.SWEEP_KERNELS["sweep_block128"]
    # 3e9 bytes in 3 ms = 1000 GB/s; frac against the peak in use
    assert abs(r["achieved"] - 1000.0) < 1e-6
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["algorithmic_bytes_per_launch"] == 3e8
    assert r["traffic"] is None


def test_roofline_of_idle_kernels_is_zero():
    ks = _ks(sweep_group8=0.0, sweep_warp=0.0, sweep_block128=0.0, sweep_block256=0.0, sweep_cluster=0.0,
             sweep_hub_acc=0.0, sweep_hub_rest=0.0)
    assert bench._roofline(ks)["achieved"] == 0.0


def test_traffic_guard_names_a_known_group():
    t = bench.NCU_TRAFFIC
    assert t["kernel"] in bench.SWEEP_KERNELS and t["bytes_per_launch"] > 0 and len(t["sha256"]) == 64


def test_reference_arm_prints_its_contract_line():
    """`bench.py --impl reference` (the oracle on the host) on a tiny stream:
    one JSON line with the reference arm's keys."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--rmat-scale", "12",
                          "--steps", "2", "--warmup", "1", "--cpu-budget", "5"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "updates/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["warmup"] == 1 and "batches 1..2" in d["cpu_baseline"]["sample"]
