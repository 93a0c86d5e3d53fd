#!/usr/bin/env python3
"""Benchmark of the g(lambda) triangular-domain mapping (arXiv:1308.1419) on one GB300.

Workload (the headline one): the mapping probe sweep.  One step = the g(lambda) probe over
every triangle side N in {1024, 4096, 16384, 65536} and block side rho in {8, 16, 32} (12
launches, chunked schedule by default); each in-domain element gets uint32
splitmix32(i N + j) in packed lower-triangular storage.  The metric is useful triangle pairs per second.  The same
sweep is also timed for BB, UTM, RB and REC (both schedules) and reported under "compare"
with the paper's improvement factor I = t_BB / t_strategy.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (the plain definition
of the probe) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIZES = [1024, 4096, 16384, 65536]
RHOS = [8, 16, 32]
STRATS = ["LTM", "BB", "UTM", "RB", "REC", "UTM-BLOCK"]
METRIC = "useful triangle pairs/s (g(lambda) probe sweep)"
UNIT = "pairs/s"

# DRAM traffic of the probe kernel (dram__bytes_read.sum + dram__bytes_write.sum), one ncu launch
# per block side at N = 65536 (the launches the roofline line reports; two 1-pass metrics), in
# bytes per launch.  The numbers hold for the kernel sources whose digest is recorded here; once
# they change the roofline line reports traffic as null until a new capture is taken.
PROBE_SOURCES = ("td_probe.cu", "td_tiles.cuh", "td_device.cuh", "td_strategies.cuh")
PROBE_TRAFFIC = {
    "sources_sha256": "99d0ef2a15609836a27a658e98bce57d1eadbbb81a39851515023b1a8bd82f2a",
    "bytes_per_launch": {8: 8540654080, 16: 8545221120, 32: 8546967552},
    "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none "
               "-k regex:k_probe_chunked -s 3 -c 1 "
               "python bench.py --case probe:LTM:chunked:65536:<rho> --steps 1 --warmup 3",
}


def tri(n):
    return n * (n + 1) // 2


def sweep_pairs():
    return sum(tri(N) for N in SIZES for _ in RHOS)


def probe_sources_digest():
    import hashlib
    h = hashlib.sha256()
    for name in PROBE_SOURCES:
        with open(os.path.join(ROOT, "paper_1308_1419_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def sweep_slice(td, N, rho, ws, rank):
    """This rank's block rows and packed slice of the triangle of side N: the td_partition share
    (the whole triangle on one rank)."""
    if ws == 1:
        return 0, -(-N // rho), 0, tri(N)
    return td.td_partition(N, rho, ws, rank)


def headline_config(sched, ws=1):
    return {"workload": f"probe sweep: N in {{1024,4096,16384,65536}} x rho in {{8,16,32}}, g(lambda), {sched} schedule",
            "useful_pairs_per_step": sweep_pairs(),
            "parallelism": "one GPU" if ws == 1 else
            f"{ws} ranks, each the td_partition block-row slice of every triangle (no data-path collective)",
            "l2": "inputs none; each step's three N=65536 launches write 8.6 GB each (> 129 MB L2), "
                  "so L2 holds nothing of the previous step"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores():
    """Host cores this process may run on (the oracle's threads use all of them)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_rate(items, seconds, threads):
    """Throughput of the CPU oracle: `threads` host threads take work items (fn, units) in turn,
    cycling through the list, until `seconds` have passed; every item is an independent call into
    the C oracle, which runs with the interpreter lock released.  Returns (units/s, units, s)."""
    import itertools
    import threading
    lock = threading.Lock()
    order = itertools.cycle(range(len(items)))
    done = [0]
    t0 = time.perf_counter()
    stop = t0 + seconds

    def worker():
        while time.perf_counter() < stop:
            with lock:
                k = next(order)
            fn, units = items[k]
            fn()
            with lock:
                done[0] += units

    pool = [threading.Thread(target=worker) for _ in range(threads)]
    for t in pool:
        t.start()
    for t in pool:
        t.join()
    dt = time.perf_counter() - t0
    return done[0] / dt, done[0], dt


def cpu_baseline_entry(items, seconds, unit, sample):
    """The oracle on one host core and on all of them (threads over disjoint work items)."""
    cores = host_cores()
    v1, u1, t1 = cpu_rate(items, seconds, 1)
    vn, un, tn = cpu_rate(items, seconds, cores)
    return {"value": vn, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample,
            "one_core": {"value": v1, "cores": 1, "units": u1, "seconds": t1},
            "all_cores": {"value": vn, "cores": cores, "units": un, "seconds": tn}}


def probe_items(rows=256):
    """Work items of the headline's CPU sample: the oracle probe on whole rows of the lower half of
    the N = 65536 triangle (rows 32768 .. 65535, `rows` at a time)."""
    import oracle
    N = 65536
    return [((lambda a=i0: oracle.probe(N, a, a + rows)), tri(i0 + rows) - tri(i0))
            for i0 in range(N // 2, N, rows)]


def cpu_oracle_sample(seconds_target=6.0):
    """The oracle probe on one core and on all cores, ~seconds_target each."""
    return cpu_baseline_entry(probe_items(), seconds_target, UNIT,
                              "whole rows of the N=65536 triangle from row 32768 on, 256 rows per work item")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle  # noqa: F401  (builds/loads the C oracle before timing)
    items = probe_items(rows=64)
    cores = host_cores()
    seconds = 1.0  # one step: about a second of all-core oracle work on whole rows of the triangle
    for _ in range(args.warmup):
        cpu_rate(items, 0.2, cores)
    pairs, dt = 0, 0.0
    for _ in range(args.steps):
        _, u, t = cpu_rate(items, seconds, cores)
        pairs += u
        dt += t
    v = pairs / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (no input; hash of (i, j))",
        "config": headline_config(args.sched),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step, about 1 s of whole rows (64 at a time) of the N=65536 triangle from "
                                   "row 32768 on, threads over disjoint rows"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1308_1419_gb300 import td

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    # Each rank's share of every triangle of the sweep: its block rows of the partition (contiguous
    # lambda ranges, contiguous packed slices; no exchange between ranks).  One rank: the whole
    # triangle through td_map_probe.
    shard = {(N, rho): sweep_slice(td, N, rho, ws, rank) for N in SIZES for rho in RHOS}
    out = torch.empty(max(4, max(o1 - o0 for _, _, o0, o1 in shard.values())), dtype=torch.int32, device=dev)

    def probe_launch(strategy, sched, N, rho, buf):
        if ws == 1:
            return td.td_map_probe(strategy, sched, N, rho, buf)[1]
        br0, br1, _, _ = shard[(N, rho)]
        if br1 <= br0:
            return {"launches": 0}
        return td.td_map_probe_rows(strategy, N, rho, br0, br1, buf)[1]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def sweep(strategy, sched, events=None):
        launches = 0
        for N in SIZES:
            for rho in RHOS:
                if events is not None:
                    events[(N, rho)][0].record(stream)
                st = probe_launch(strategy, sched, N, rho, out)
                if events is not None:
                    events[(N, rho)][1].record(stream)
                launches += st["launches"]
        return launches

    def timed(strategy, sched, steps, warmup, per_launch=False):
        for _ in range(warmup):
            sweep(strategy, sched)
        evs_all = []
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        launches = 0
        for _ in range(steps):
            evs = None
            if per_launch:
                evs = {(N, r): (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for N in SIZES for r in RHOS}
                evs_all.append(evs)
            launches += sweep(strategy, sched, evs)
        t1.record(stream)
        barrier()
        ms = t0.elapsed_time(t1)
        per = {}
        if per_launch:
            for key in evs_all[0]:
                per[key] = [e[key][0].elapsed_time(e[key][1]) for e in evs_all]
        return ms, launches, per

    # ---- headline: g(lambda) sweep
    with ClockSampler(local) as clk:
        ms, launches, per = timed("LTM", args.sched, args.steps, args.warmup, per_launch=True)
    ms_t = torch.tensor([ms], device=dev)
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms = float(ms_t.item())
    units = sweep_pairs() * args.steps  # every rank has its share of the same sweep
    value = units / (ms / 1e3)

    # ---- compared strategies (same sweep), both schedules
    compare = {}
    for strategy in ([] if args.no_compare or ws > 1 else STRATS):
        for sched in (("chunked", "persistent", "grid") if strategy in ("LTM", "BB", "REC", "UTM-BLOCK")
                      else ("persistent", "grid")):
            csteps = max(3, min(20, args.steps // 2))
            cms, _, cper = timed(strategy, sched, csteps, 2, per_launch=True)
            compare[f"{strategy}/{sched}"] = {
                "pairs_per_s": sweep_pairs() * csteps / (cms / 1e3),
                "ms_N65536": {str(r): statistics.median(cper[(65536, r)]) for r in RHOS},
            }
    bb = compare["BB/grid"]["ms_N65536"] if compare else {}
    for key, c in compare.items():
        c["I_vs_BB_grid_N65536"] = {r: bb[r] / c["ms_N65536"][r] for r in bb}
        same = compare.get("BB/" + key.split("/")[1])
        if same:
            c["I_vs_BB_same_schedule_N65536"] = {r: same["ms_N65536"][r] / c["ms_N65536"][r] for r in bb}

    # ---- write-only reference: cudaMemsetAsync of the same 8.6 GB (not a roofline denominator;
    # skipped with --no-compare so that a profiler's launch list holds only the timed step's kernels)
    memset_gbps = None
    if not args.no_compare and ws == 1:
        for _ in range(3):
            out.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            out.zero_()
        e1.record(stream)
        torch.cuda.synchronize()
        memset_gbps = 5 * out.numel() * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9

    # ---- roofline of the dominant kernel: g(lambda) probe launches at N = 65536
    peak, peak_kind = load_peaks()
    per_rho = {}
    for r in RHOS:
        t = statistics.mean(per[(65536, r)])
        _, _, o0, o1 = shard[(65536, r)]
        per_rho[r] = {"ms": t, "GBps": 4 * (o1 - o0) / (t / 1e3) / 1e9}
    dom = max(RHOS, key=lambda r: per_rho[r]["ms"])
    achieved = per_rho[dom]["GBps"]
    traffic, traffic_note = None, "no ncu capture recorded for these kernel sources"
    if (args.sched == "chunked" and PROBE_TRAFFIC["sources_sha256"] == probe_sources_digest()
            and dom in PROBE_TRAFFIC["bytes_per_launch"]):
        traffic = PROBE_TRAFFIC["bytes_per_launch"][dom]
        traffic_note = "ncu dram__bytes_read.sum + dram__bytes_write.sum of one N=65536 launch at this rho"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_note": traffic_note, "kernel": f"g(lambda) probe, {args.sched} schedule, rho={dom}, N=65536",
                "memset_write_GBps": memset_gbps,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs, copy)" if peak_kind == "measured" else "fallback",
                "per_rho": {str(r): v for r, v in per_rho.items()},
                "algorithmic_bytes_per_launch": 4 * (shard[(65536, dom)][3] - shard[(65536, dom)][2])}

    # ---- end to end: the same sweep through the public API with the output in HOST memory.
    # Three ways: (copy) the kernel writes device memory and the result is copied to pinned host
    # memory; (direct) the kernel writes the pinned host buffer itself over the host link;
    # (overlap) copies on a second stream overlap the next launch.  The fastest is reported; all
    # are kept in the line.
    e2e = None
    if not args.no_e2e:
        host = torch.empty(out.numel(), dtype=torch.int32, pin_memory=True)
        d2h = sum(4 * tri(N) for N in SIZES for _ in RHOS)  # all ranks' slices: the whole sweep
        e2e_steps = max(2, min(5, args.steps // 4))

        def size(N, rho):
            return shard[(N, rho)][3] - shard[(N, rho)][2]

        def e2e_copy():
            for N in SIZES:
                for rho in RHOS:
                    probe_launch("LTM", args.sched, N, rho, out)
                    host[: size(N, rho)].copy_(out[: size(N, rho)], non_blocking=True)

        def e2e_direct():
            for N in SIZES:
                for rho in RHOS:
                    probe_launch("LTM", args.sched, N, rho, host)

        # (overlap) the kernel writes one of two device buffers while the previous result goes to
        # pinned host memory on a copy stream: the host link (~190 GB/s here) is the bound
        slots = [out, torch.empty_like(out)]
        copy_stream = torch.cuda.Stream()
        slot_free = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_overlap():
            k = 0
            for N in SIZES:
                for rho in RHOS:
                    slot = slots[k % 2]
                    stream.wait_event(slot_free[k % 2])
                    probe_launch("LTM", args.sched, N, rho, slot)
                    copy_stream.wait_stream(stream)
                    with torch.cuda.stream(copy_stream):
                        host[: size(N, rho)].copy_(slot[: size(N, rho)], non_blocking=True)
                        slot_free[k % 2].record(copy_stream)
                    k += 1
            stream.wait_stream(copy_stream)

        modes = {}
        for name, fn in (("copy", e2e_copy), ("direct", e2e_direct), ("overlap", e2e_overlap)):
            fn()
            barrier()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                fn()
            torch.cuda.synchronize()
            dt_t = torch.tensor([time.perf_counter() - t0], device=dev)
            if dist is not None:
                dist.all_reduce(dt_t, op=dist.ReduceOp.MAX)
            modes[name] = sweep_pairs() * e2e_steps / float(dt_t.item())
        best = max(modes, key=modes.get)
        e2e = {"value": modes[best], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
               "mode": best, "modes": modes}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample()

    configs = None
    if rank == 0 and ws == 1 and not args.no_configs:
        configs = run_configs(args, td, stream)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic (no input array; each pair writes a hash of (i, j))",
            "config": headline_config(args.sched, ws),
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "compare": compare,
            "configs": configs,
        }), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def load_peak_table():
    """MEASURED_PEAKS.json as written on the box (copy GB/s, BF16 TF/s burst and sustained, SM clock)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def alu_peak_ops(torch):
    """FP32 / INT32 issue peak: SMs x 128 lanes x the maximum SM clock (an FMA counts once)."""
    table, _ = load_peak_table()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = float(table.get("sm_max_mhz", 2070.0))
    return sms * 128 * mhz * 1e6, f"{sms} SMs x 128 lanes x {mhz:.0f} MHz"


def _events_ms(torch, stream, fn, reps, warmup=3):
    """Mean device time of fn() over `reps` back-to-back calls, CUDA events on `stream`."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _rel_err(got, want):
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    rel = np.abs(got - want) / np.maximum(want, 1e-30)
    rel[want == 0] = np.abs(got[want == 0])
    return {"max_rel": float(rel.max()), "rms_rel": float(np.sqrt((rel ** 2).mean())), "pairs": int(want.size)}


def run_configs(args, td, stream):
    """The other workloads of the method, each timed by CUDA events in this run, with its roofline,
    a sampled check against the oracle and the oracle's own throughput on the host cores:
    plain EDM (n = 2048, d = 3, and n = 8192, 32768), the collision table (n = 32768), the precision
    form (BF16 Gram vs FP32 direct, n = 16384, d = 256) and the batched form (512 problems)."""
    import numpy as np
    import torch

    import oracle
    from paper_1308_1419_gb300 import synth

    peaks, peak_kind = load_peak_table()
    copy = float(peaks["hbm_gbs"])
    alu, alu_how = alu_peak_ops(torch)
    cpu_s = 1.0 if not args.no_cpu else 0.0
    configs = {}

    def cpu_entry(items, sample):
        return cpu_baseline_entry(items, cpu_s, UNIT, sample) if cpu_s > 0 else None

    # ---- 1. plain EDM: n = 2048, d = 3, rho = 16 (launch-bound: the 8.4 MB output sits in L2), then
    # the store-bound sizes n = 8192 and 32768 (outputs of 134 MB and 2.1 GB, beyond L2)
    xh = synth.plain_edm()
    x = torch.from_numpy(xh).cuda()
    n = xh.shape[0]
    out = torch.empty(tri(32768), dtype=torch.float32, device="cuda")
    ms = {}
    for strat in ("LTM", "BB"):
        for sched in ("grid", "persistent", "chunked"):
            ms[f"{strat}/{sched}"] = _graph_ms(lambda: td.td_edm(strat, sched, x, 16, out), 20)
    best = min((k for k in ms if k.startswith("LTM/")), key=ms.get)
    got, _ = td.td_edm(best.split("/")[0], best.split("/")[1], x, 16, out)
    err = _rel_err(got[: tri(n)].cpu().numpy(), oracle.edm(xh))
    sweep = {}
    for nn in (8192, 32768):
        xs = torch.from_numpy(synth.uniform_points(nn, 3, synth.seed_for(1))).cuda()
        row = {}
        for strat in ("LTM", "BB"):
            row[f"{strat}/chunked/16"] = _events_ms(torch, stream, lambda: td.td_edm(strat, "chunked", xs, 16, out), 10)
            row[f"{strat}/persistent/128"] = _events_ms(
                torch, stream, lambda: td.td_edm(strat, "persistent", xs, 128, out), 10)
        ltm_best = min((k for k in row if k.startswith("LTM/")), key=row.get)
        bb_best = min((k for k in row if k.startswith("BB/")), key=row.get)
        gbps = 4 * tri(nn) / (row[ltm_best] / 1e3) / 1e9
        sweep[str(nn)] = {"ms": row, "best_LTM": ltm_best, "pairs_per_s": tri(nn) / (row[ltm_best] / 1e3),
                          "I_best_BB_over_best_LTM": row[bb_best] / row[ltm_best],
                          "roofline": {"bound": "hbm", "achieved": gbps, "peak": copy, "unit": "GB/s",
                                       "frac": gbps / copy}}
    rows = 64
    configs["plain_edm"] = {
        "workload": "EDM n=2048, d=3, x ~ U[0,1)^3 (seed 1309), rho=16; each schedule replayed 20x in a CUDA graph "
                    "(output 8.4 MB, L2-resident: launch-bound); store-bound sizes n=8192, 32768 below",
        "pairs": tri(n), "ms": ms, "best_LTM": best, "pairs_per_s": tri(n) / (ms[best] / 1e3),
        "I_vs_BB_same_schedule": {sc: ms[f"BB/{sc}"] / ms[f"LTM/{sc}"] for sc in ("grid", "persistent", "chunked")},
        "roofline": {"bound": "hbm", "achieved": 4 * tri(n) / (ms[best] / 1e3) / 1e9, "peak": copy, "unit": "GB/s",
                     "frac": 4 * tri(n) / (ms[best] / 1e3) / 1e9 / copy,
                     "note": "L2-resident output; the n=32768 entry of 'sweep' is the HBM roofline case"},
        "error_vs_fp64_oracle": err, "tolerance": 2e-6,
        "sweep": sweep,
        "cpu_baseline": cpu_entry([((lambda a=i0: oracle.edm(xh, a, min(a + rows, n))),
                                    tri(min(i0 + rows, n)) - tri(i0)) for i0 in range(0, n, rows)],
                                  "the FP64 oracle distance map of this n=2048 input, 64 whole rows per work item"),
    }

    # ---- 3. collision table: n = 32768 spheres (FP32/INT32 issue-bound: 9 operations per pair)
    c, r = synth.spheres()
    ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
    nc = r.size
    table = torch.empty(td.td_collide_words(nc), dtype=torch.int32, device="cuda")
    cms = {}
    for strat in ("LTM", "BB"):
        for sched in ("grid", "persistent"):
            cms[f"{strat}/{sched}"] = _events_ms(torch, stream, lambda: td.td_collide(strat, sched, ct, rt, table), 20)
    cbest = min((k for k in cms if k.startswith("LTM/")), key=cms.get)
    td.td_collide(cbest.split("/")[0], cbest.split("/")[1], ct, rt, table)
    rng = np.random.default_rng(7)
    ii = rng.integers(1, nc, 200000).astype(np.uint32)
    jj = (rng.random(ii.size) * ii).astype(np.uint32)
    words = table.cpu().numpy().view(np.uint32)
    bi, bj = ii.astype(np.int64) // 32, jj.astype(np.int64) // 32
    w = 32 * (bi * (bi + 1) // 2 + bj) + ii % 32
    gbits = (words[w] >> (jj % 32).astype(np.uint32)) & 1
    pairs_c = nc * (nc - 1) // 2
    ops = 9 * pairs_c / (cms[cbest] / 1e3)
    groups = [(np.ascontiguousarray(c[g:g + 2048]), np.ascontiguousarray(r[g:g + 2048])) for g in range(0, nc, 2048)]
    configs["collision"] = {
        "workload": "collision table n=32768, centres int32 U[0,2^20)^3, radii U[256,2048] (seed 1311), 32x32 bit tiles",
        "pairs": pairs_c, "ms": cms, "best_LTM": cbest, "pairs_per_s": pairs_c / (cms[cbest] / 1e3),
        "I_vs_BB_same_schedule": {sc: cms[f"BB/{sc}"] / cms[f"LTM/{sc}"] for sc in ("grid", "persistent")},
        "roofline": {"bound": "alu", "achieved": ops, "peak": alu, "unit": "op/s", "frac": ops / alu,
                     "ops_per_pair": 9, "peak_how": alu_how},
        "sampled_pairs_bit_exact": bool(np.array_equal(gbits.astype(np.uint8), oracle.collide_pairs(c, r, ii, jj))),
        "sampled_pairs": int(ii.size),
        "cpu_baseline": cpu_entry([((lambda g=g: oracle.collide(g[0], g[1])), tri(2047)) for g in groups],
                                  "the 128-bit oracle table of 2048-sphere groups of this input, one group per "
                                  "work item"),
    }
    del table

    # ---- 4. precision form: BF16 Gram on tcgen05 + FP32 recompute, against the FP32 direct kernel
    xp_h = synth.clustered_points()
    np_, dp = xp_h.shape
    xp = torch.from_numpy(xp_h).cuda()
    outp = torch.empty(tri(np_), dtype=torch.float32, device="cuda")
    wsg = torch.empty(td.td_edm_gram_workspace(np_, dp) + 1024, dtype=torch.uint8, device="cuda")
    t_gram = _events_ms(torch, stream, lambda: td.td_edm_gram(xp, outp, wsg), 10)
    fallback = td.td_edm_gram_status(wsg)
    ii = rng.integers(0, np_, 20000).astype(np.uint32)
    jj = (rng.random(ii.size) * (ii.astype(np.float64) + 1)).astype(np.uint32)
    pos = torch.from_numpy(ii.astype(np.int64) * (ii.astype(np.int64) + 1) // 2 + jj).cuda()
    want = oracle.edm_pairs(xp_h, ii, jj)
    gram_err = _rel_err(outp[pos].cpu().numpy(), want)
    t_direct = _events_ms(torch, stream, lambda: td.td_edm("LTM", "persistent", xp, 128, outp), 5)
    direct_err = _rel_err(outp[pos].cpu().numpy(), want)
    gbps = 4 * tri(np_) / (t_gram / 1e3) / 1e9
    tflops = 2 * dp * tri(np_) / (t_gram / 1e3) / 1e12
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    chunks = [(ii[k:k + 4096], jj[k:k + 4096]) for k in range(0, ii.size, 4096)]
    configs["precision"] = {
        "workload": "EDM n=16384, d=256, 64 Gaussian clusters (sigma 0.05, seed 1312); BF16 Gram on tcgen05 with "
                    "FP32 accumulate + FP32 direct recompute where D^2 < 1e-2 (|x|^2 + |y|^2)",
        "pairs": tri(np_), "ms": {"gram_bf16": t_gram, "direct_fp32_LTM_rho128": t_direct},
        "pairs_per_s": tri(np_) / (t_gram / 1e3), "speedup_vs_direct_fp32": t_direct / t_gram,
        "recomputed_pairs": fallback, "recomputed_fraction": fallback / tri(np_),
        "error_vs_fp64_oracle": {"gram": gram_err, "direct_fp32": direct_err},
        "roofline": {"bound": "hbm", "achieved": gbps, "peak": copy, "unit": "GB/s", "frac": gbps / copy,
                     "note": "output bytes of the whole form (main pass + recompute) over its time"},
        "tensor": {"achieved_tflops": tflops, "peak_tflops": bf16, "frac": tflops / bf16,
                   "flops": "2 d per pair of the triangle"},
        "direct_alu": {"achieved": 2 * dp * tri(np_) / (t_direct / 1e3), "peak": alu,
                       "frac": 2 * dp * tri(np_) / (t_direct / 1e3) / alu, "unit": "op/s"},
        "cpu_baseline": cpu_entry([((lambda a=a, b=b: oracle.edm_pairs(xp_h, a, b)), a.size) for a, b in chunks],
                                  "the FP64 oracle distance of 4096 random pairs of this input per work item"),
    }
    del outp, wsg

    # ---- 5. batched form: 512 problems in one persistent launch, against one launch per problem
    ns, ds, xb_h = synth.batched_problems()
    xb = torch.from_numpy(xb_h).cuda()
    xs_, os_ = td.batched_sizes(ns, ds)
    outb = torch.empty(os_, dtype=torch.float32, device="cuda")
    wsb = torch.empty(td.td_edm_batched_workspace(len(ns)), dtype=torch.uint8, device="cuda")
    (rho_t, cps_t), tune_ms = td.td_edm_batched_autotune(ns, ds, xb, outb, wsb)
    total = td.td_edm_batched_plan(ns, ds, rho_t, wsb)
    bms = {"one_launch": _events_ms(torch, stream,
                                    lambda: td.td_edm_batched_run(len(ns), rho_t, total, xb, outb, wsb, cps_t), 5)}
    bms["one_launch_graph"] = _graph_ms(lambda: td.td_edm_batched_run(len(ns), rho_t, total, xb, outb, wsb, cps_t), 5)
    xo, oo = [0], [0]
    for nq, dq in zip(ns, ds):
        xo.append(xo[-1] + int(nq) * int(dq))
        oo.append(oo[-1] + tri(int(nq)))
    # per-problem buffers of their own: td_edm wants 16-byte-aligned points and output
    xs_l = [xb[xo[p]: xo[p + 1]].view(int(ns[p]), int(ds[p])).clone() for p in range(len(ns))]
    outs_l = [torch.empty(oo[p + 1] - oo[p], dtype=torch.float32, device="cuda") for p in range(len(ns))]

    def per_problem():
        for p in range(len(ns)):
            td.td_edm("LTM", "persistent", xs_l[p], 128, outs_l[p])
    bms["per_problem"] = _events_ms(torch, stream, per_problem, 3, warmup=1)
    bms["per_problem_graph"] = _graph_ms(per_problem, 3)
    td.td_edm_batched_run(len(ns), rho_t, total, xb, outb, wsb, cps_t)
    torch.cuda.synchronize()
    order = np.argsort(ns, kind="stable")
    check = list(order[:4]) + [p for p in order if ds[p] == 64 and 1000 < ns[p] < 2000][:2]
    errs = [_rel_err(outb[oo[p]: oo[p + 1]].cpu().numpy(),
                     oracle.edm(xb_h[xo[p]: xo[p + 1]].reshape(int(ns[p]), int(ds[p])))) for p in check]
    ops_b = sum(2 * int(dq) * tri(int(nq)) for nq, dq in zip(ns, ds))
    tb = bms["one_launch"]
    items = []
    for p in range(len(ns)):
        nq, dq = int(ns[p]), int(ds[p])
        step = max(1, (1 << 18) // max(nq, 1))
        xq = xb_h[xo[p]: xo[p + 1]].reshape(nq, dq)
        for i0 in range(0, nq, step):
            i1 = min(i0 + step, nq)
            items.append(((lambda xq=xq, a=i0, b=i1: oracle.edm(xq, a, b)), tri(i1) - tri(i0)))
    perm = np.random.default_rng(1313).permutation(len(items))
    configs["batched"] = {
        "workload": "512 EDM problems, n = floor(64 * 128^U) in [64, 8192], d from {3, 16, 64}, x ~ U[0,1) "
                    "(seed 1313); one persistent launch (prefix-sum search, then g) vs one td_edm launch per problem",
        "pairs": os_, "autotuned": {"rho": rho_t, "ctas_per_sm": cps_t, "ms": tune_ms}, "ms": bms,
        "pairs_per_s": os_ / (tb / 1e3),
        "speedup_vs_per_problem": bms["per_problem"] / tb,
        "speedup_vs_per_problem_graph": bms["per_problem_graph"] / tb,
        "roofline": {"bound": "alu", "achieved": ops_b / (tb / 1e3), "peak": alu, "unit": "op/s",
                     "frac": ops_b / (tb / 1e3) / alu, "ops": "2 d_p FP32 instructions per pair", "peak_how": alu_how},
        "error_vs_fp64_oracle": {"problems_checked": [int(p) for p in check],
                                 "max_rel": max(e["max_rel"] for e in errs)},
        "cpu_baseline": cpu_entry([items[k] for k in perm],
                                  "the FP64 oracle distance map over row ranges (~2^18 pairs each) of the batch's "
                                  "problems, in a seeded random order so that any prefix mixes the three d"),
    }
    configs["peaks"] = {"copy_GBps": copy, "bf16_tflops": float(peaks.get("bf16_tflops", 0.0)), "alu_ops": alu,
                        "kind": peak_kind}
    return configs


def run_case(args):
    """One kernel alone: W warm-up launches, then K timed launches (for profilers and sweeps)."""
    import torch
    from paper_1308_1419_gb300 import td
    from paper_1308_1419_gb300 import synth
    for opt in args.opt:
        name, value = opt.split("=")
        td.td_set_option(name, int(value))
    parts = args.case.split(":")
    kind, strategy, sched = (parts + ["", ""])[:3]
    if kind == "probe":
        N, rho = int(parts[3]), int(parts[4])
        out = torch.empty(tri(N), dtype=torch.int32, device="cuda")
        pairs, nbytes = tri(N), 4 * tri(N)
        def call():
            td.td_map_probe(strategy, sched, N, rho, out)
    elif kind == "edm":
        # edm:<strategy>:<sched>:<n>:<d>:<rho>[:x2]  (x2: the library option that turns the packed
        # f32x2 arithmetic of the tiled kernel on; same results)
        n, d, rho = int(parts[3]), int(parts[4]), int(parts[5])
        if len(parts) > 6 and parts[6] == "x2":
            td.td_set_option("edm_f32x2", 1)
        if n == 16384 and d == 256:
            xh = synth.clustered_points()
        else:
            xh = synth.uniform_points(n, d, synth.seed_for(1))
        x = torch.from_numpy(xh).cuda()
        out = torch.empty(tri(n), dtype=torch.float32, device="cuda")
        pairs, nbytes = tri(n), 4 * tri(n)
        def call():
            td.td_edm(strategy, sched, x, rho, out)
    elif kind == "collide":
        n = int(parts[3])
        c, r = synth.spheres(n)
        ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
        table = torch.empty(td.td_collide_words(n), dtype=torch.int32, device="cuda")
        pairs, nbytes = n * (n - 1) // 2, 4 * td.td_collide_words(n)
        def call():
            td.td_collide(strategy, sched, ct, rt, table)
    elif kind == "edmstrict":
        # edmstrict:<n>:<d>[:<strategy>:<rho>]: strict-lower distance map, element-level strict g,
        # or (with a strategy) mapped at the block level over the triangle of side n - 1
        n, d = int(strategy), int(sched)
        x = torch.from_numpy(synth.uniform_points(n, d, synth.seed_for(1))).cuda()
        out = torch.empty(max(n * (n - 1) // 2, 4), dtype=torch.float32, device="cuda")
        pairs, nbytes = n * (n - 1) // 2, 4 * (n * (n - 1) // 2)
        if len(parts) > 4:
            def call():
                td.td_edm_strict_blocks(parts[3], x, int(parts[4]), out)
        else:
            def call():
                td.td_edm_strict(x, out)
    elif kind == "collidestrict":
        # collidestrict:<n>[:<strategy>:<rho>]: strict-lower collision bits, element-level strict g,
        # or (with a strategy) mapped at the block level
        n = int(strategy)
        c, r = synth.spheres(n)
        ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
        bits = torch.empty(max(td.td_collide_strict_words(n), 4), dtype=torch.int32, device="cuda")
        pairs, nbytes = n * (n - 1) // 2, 4 * td.td_collide_strict_words(n)
        if len(parts) > 3:
            def call():
                td.td_collide_strict_blocks(parts[2], ct, rt, int(parts[3]), bits)
        else:
            def call():
                td.td_collide_strict(ct, rt, bits)
    elif kind == "gram":
        # gram:<n>:<d>: BF16 tensor-core Gram form with FP32 direct recompute
        n, d = int(strategy), int(sched)
        xh = synth.clustered_points() if (n, d) == (16384, 256) else synth.uniform_points(n, d, synth.seed_for(4))
        x = torch.from_numpy(xh).cuda()
        out = torch.empty(tri(n), dtype=torch.float32, device="cuda")
        ws = torch.empty(td.td_edm_gram_workspace(n, d) + 1024, dtype=torch.uint8, device="cuda")
        pairs, nbytes = tri(n), 4 * tri(n)
        def call():
            td.td_edm_gram(x, out, ws)
    elif kind == "batched":
        # batched:<how>:<rho>:<ctas_per_sm>[:<nprob>], how = one (single persistent launch), graph (its
        # graph replay), per (one td_edm launch per problem), pergraph (those launches as one graph),
        # tune (autotuned one launch); nprob: the first problems of the 512-problem batch's recipe
        # (default all 512)
        how, rho, cps = strategy, int(sched), int(parts[3])
        nprob = int(parts[4]) if len(parts) > 4 else 512
        ns, ds, xh = synth.batched_problems(nprob=nprob)
        x = torch.from_numpy(xh).cuda()
        xs, os_ = td.batched_sizes(ns, ds)
        out = torch.empty(os_, dtype=torch.float32, device="cuda")
        ws = torch.empty(td.td_edm_batched_workspace(len(ns)), dtype=torch.uint8, device="cuda")
        pairs, nbytes = os_, 4 * os_
        if how == "tune":
            (rho, cps), _ = td.td_edm_batched_autotune(ns, ds, x, out, ws)
            print(json.dumps({"autotuned": {"rho": rho, "ctas_per_sm": cps}}), flush=True)
        total = td.td_edm_batched_plan(ns, ds, rho, ws)
        if how in ("one", "tune"):
            def call():
                td.td_edm_batched_run(len(ns), rho, total, x, out, ws, cps)
        elif how == "graph":
            td.td_edm_batched_run(len(ns), rho, total, x, out, ws, cps)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                td.td_edm_batched_run(len(ns), rho, total, x, out, ws, cps)
            def call():
                graph.replay()
        else:
            # per: one td_edm launch per problem; pergraph: the same launches replayed as one graph
            xo = [0]
            oo = [0]
            for n, d in zip(ns, ds):
                xo.append(xo[-1] + int(n) * int(d))
                oo.append(oo[-1] + int(n) * (int(n) + 1) // 2)
            xs_l = [x[xo[p]: xo[p + 1]].view(int(ns[p]), int(ds[p])).clone() for p in range(len(ns))]
            outs = [torch.empty(oo[p + 1] - oo[p], dtype=torch.float32, device="cuda") for p in range(len(ns))]
            def per_problem():
                for p in range(len(ns)):
                    td.td_edm("LTM", "persistent", xs_l[p], rho, outs[p])
            if how == "pergraph":
                per_problem()
                torch.cuda.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    per_problem()
                def call():
                    graph.replay()
            else:
                call = per_problem
    else:
        raise SystemExit(f"unknown case {args.case}")
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    for k in range(args.steps):
        ev[2 * k].record()
        call()
        ev[2 * k + 1].record()
    torch.cuda.synchronize()
    ms = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)]
    med = statistics.median(ms)
    print(json.dumps({"case": args.case, "ms_median": med, "ms_min": min(ms),
                      "pairs_per_s": pairs / (med / 1e3), "GBps_written": nbytes / (med / 1e3) / 1e9}), flush=True)


def run_feature_sweep(args):
    """The distance-map figure of Sec. IV: N = 1024 k (k = 1 .. 30), d = 1 .. 4, rho = 16, every
    strategy under one schedule; per (d, N) the mean launch time over a replayed graph of `steps`
    launches, and I = t_BB / t_strategy."""
    import torch
    from paper_1308_1419_gb300 import synth, td

    sched = args.sched
    sizes = [1024 * k for k in range(1, 31)]
    strats = ["LTM", "BB", "RB", "REC", "UTM"] if sched != "chunked" else ["LTM", "BB", "REC"]
    out = torch.empty(tri(max(sizes)), dtype=torch.float32, device="cuda")
    table = {}
    steps = max(3, min(10, args.steps))
    for d in (1, 2, 3, 4):
        xs = torch.from_numpy(synth.uniform_points(max(sizes), d, synth.seed_for(1) + d)).cuda()
        per = {s: [] for s in strats}
        for N in sizes:
            x = xs[:N]
            for strategy in strats:
                # `steps` launches captured in one graph, so small launches are timed on the GPU and
                # not by the host's call overhead
                td.td_edm(strategy, sched, x, 16, out)
                torch.cuda.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    for _ in range(steps):
                        td.td_edm(strategy, sched, x, 16, out)
                graph.replay()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                graph.replay()
                e1.record()
                torch.cuda.synchronize()
                per[strategy].append(e0.elapsed_time(e1) / steps)
        table[str(d)] = {"ms": per, "I_vs_BB": {s: [b / t for b, t in zip(per["BB"], per[s])] for s in strats}}
    print(json.dumps({"sweep": "EDM features (Sec. IV)", "rho": 16, "schedule": sched, "N": sizes, "steps": steps,
                      "data": "synthetic U[0,1)^d", "by_d": table}), flush=True)


def _graph_ms(fn, steps):
    """Mean device time of fn() over `steps` launches captured in one CUDA graph."""
    import torch
    fn()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(steps):
            fn()
    graph.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    graph.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_ltm_variant_sweep(args):
    """The LTM implementation comparison of Sec. III-A: the map-only dummy kernel, and the probe
    body, under BB and under each evaluation of g (exact fix-up, LTM-X, LTM-N rounded per
    operation and contracted into fused multiply-adds, LTM-R),
    N = 1024 k (k = 1 .. 30), rho = 16, paper-style GRID launch; I = t_BB / t_variant.  Also each
    variant's first failing lambda below 2^32 (the exact g has none)."""
    import torch
    from paper_1308_1419_gb300 import td

    sizes = [1024 * k for k in range(1, 31)]
    maps = ["BB", "LTM", "LTM-X", "LTM-N", "LTM-N-FMA", "LTM-R"]
    sched = args.sched if args.sched != "chunked" else "grid"
    steps = max(3, min(10, args.steps))
    sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(tri(max(sizes)), dtype=torch.int32, device="cuda")
    ms = {m: [_graph_ms(lambda: td.td_map_dummy(m, sched, N, 16, sink), steps) for N in sizes] for m in maps}
    ms_probe = {m: [_graph_ms(lambda: td.td_map_probe(m, sched, N, 16, out), steps) for N in sizes] for m in maps}
    first = {}
    for m in maps[1:]:
        r = td.td_ltm_variant_check(m, 0, 1 << 32).cpu().tolist()
        first[m] = {"failures_below_2^32": int(r[0]), "first_failing_lambda": None if r[0] == 0 else int(r[1])}
    print(json.dumps({"sweep": "LTM implementations (Sec. III-A), map-only dummy kernel", "rho": 16, "schedule": sched,
                      "N": sizes, "steps": steps, "ms": ms,
                      "I_vs_BB": {m: [b / t for b, t in zip(ms["BB"], ms[m])] for m in maps},
                      "mean_I_vs_BB": {m: statistics.mean(b / t for b, t in zip(ms["BB"], ms[m])) for m in maps},
                      "probe_ms": ms_probe,
                      "probe_mean_I_vs_BB": {m: statistics.mean(b / t for b, t in zip(ms_probe["BB"], ms_probe[m]))
                                             for m in maps},
                      "first_failure": first}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-compare", action="store_true", help="skip the BB/UTM/RB/REC comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (plain EDM, collision, precision, batched)")
    ap.add_argument("--sched", default="chunked", choices=["chunked", "persistent", "grid"],
                    help="schedule of the headline g(lambda) sweep")
    ap.add_argument("--sweep", default=None, choices=["edm-features", "ltm-variants"],
                    help="edm-features: the distance-map sweep of Sec. IV (N = 1024..30720, d = 1..4, rho 16, "
                         "all strategies under --sched); ltm-variants: the LTM implementations of Sec. III-A "
                         "against BB with the map-only dummy kernel; one JSON line")
    ap.add_argument("--opt", action="append", default=[],
                    help="library option for --case runs, name=value (edm_f32x2, probe_strip); repeatable")
    ap.add_argument("--case", default="sweep",
                    help="sweep (default), or one kernel alone: probe:<strategy>:<sched>:<N>:<rho>, "
                         "edm:<strategy>:<sched>:<n>:<d>:<rho>, collide:<strategy>:<sched>:<n>")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.sweep == "edm-features":
        run_feature_sweep(args)
    elif args.sweep == "ltm-variants":
        run_ltm_variant_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.case != "sweep":
        run_case(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
