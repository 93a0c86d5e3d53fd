"""bench.py on the CPU: its helpers, and the reference arm (the oracle timed on host cores)
end to end, printing the contract's JSON line."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_helpers():
    assert bench.tri(65536) == 65536 * 65537 // 2
    assert bench.sweep_pairs() == 3 * sum(n * (n + 1) // 2 for n in bench.SIZES)
    cfg = bench.headline_config("chunked")
    assert cfg["useful_pairs_per_step"] == bench.sweep_pairs() and "chunked" in cfg["workload"]
    assert len(bench.probe_sources_digest()) == 64


def test_reference_arm_prints_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"] == bench.headline_config("chunked")


def test_cpu_rate_counts_every_item_it_ran():
    """The host-core timer of the oracle baselines: each thread takes whole work items, and the
    units reported are the sum of the items that ran, over the wall time of all threads."""
    import threading
    ran, lock = [], threading.Lock()

    def item(k):
        def fn():
            with lock:
                ran.append(k)
        return fn, k + 1

    v, units, dt = bench.cpu_rate([item(k) for k in range(5)], 0.05, 3)
    assert units == sum(k + 1 for k in ran) and units > 0 and dt >= 0.05 and v == units / dt
    e = bench.cpu_baseline_entry(bench.probe_items(rows=64)[:4], 0.05, "pairs/s", "sample")
    assert e["cores"] == bench.host_cores() and e["all_cores"]["cores"] == e["cores"]
    assert e["one_core"]["cores"] == 1 and e["value"] == e["all_cores"]["value"] > 0


def test_sweep_shards_cover_each_triangle_once():
    """bench.py --gpus N: rank r computes its td_partition slice of every triangle of the sweep, so
    the ranks' slices are disjoint, contiguous and add up to the whole sweep (strong scaling)."""
    from paper_1308_1419_gb300.build import build_libtd
    build_libtd()
    from paper_1308_1419_gb300 import td
    for ws in (1, 2, 3, 8):
        for N in bench.SIZES:
            for rho in bench.RHOS:
                parts = [bench.sweep_slice(td, N, rho, ws, r) for r in range(ws)]
                assert parts[0][2] == 0 and parts[-1][3] == bench.tri(N)
                for a, b in zip(parts, parts[1:]):
                    assert a[1] == b[0] and a[3] == b[2]
