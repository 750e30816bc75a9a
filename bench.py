#!/usr/bin/env python
"""Benchmark of the k-core hot path on GB300; prints ONE JSON line.

Default workload: the social-graph stand-in, R-MAT scale 24 with edge factor
32 and (a, b, c) = (0.45, 0.22, 0.22), symmetrised and deduplicated, plus a
planted G(5000, 0.5) core (n = 16,777,216, m = 542,922,765; int64 row_ptr);
the sweep knobs are picked by the library's autotuner first and every run is
a replayed CUDA graph.  A step is one pass of the whole path over the graph
whose raw edge samples are already resident in HBM: device CSR cleaning
(kcore_create_coo), estimate initialisation, the persistent sweep kernel until
the frontier is empty, and the int32 coreness written to a device buffer
(kcore_run).  value = undirected edges m of the cleaned graph per second of
step time.

Also reported: the same metric end to end through the C ABI with host
buffers (pinned host -> device copy of the samples and device -> host copy of
the coreness inside the timed region), the decomposition alone on the
resident graph (the paper's timing: load excluded, setup included), the sweep
kernel's roofline fraction against the measured HBM copy bandwidth, the
oracle's Batagelj-Zaversnik peel of the whole graph on one host core (its
host CSR build timed apart), SM clocks sampled during the timed region, and
`stream`: the batching / serving workload (20,000 graphs, n log-uniform in
[100, 200000], ER / R-MAT / damaged grid) as batched graphs/s and p50/p99
latency of the continuous-batching engine against one create + run per
graph, both served for real under the same Poisson arrivals, every result
compared with the oracle.

--impl reference times the oracle (plain C Batagelj-Zaversnik over its own
host CSR) on the host cores on the same workload and metric.

Launch: python bench.py [--gpus 1] [--steps K] [--warmup W] [--workload NAME];
for N > 1 under torch.distributed.run, each rank decomposes its own copy of
the workload (independent replicas, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decomposed edges/s"
UNIT = "edges/s"
L2_FLUSH_BYTES = 512 << 20
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="rmat24_planted",
                    help="er10k | road2048 | rmat22 | rmat24_planted | stream (the stream alone)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=30.0,
                    help="oracle time the CPU baseline may take per timed pass (whole graph "
                         "when one peel fits; else a prefix of the samples)")
    ap.add_argument("--ref-budget-s", type=float, default=100.0,
                    help="reference arm: timed oracle peels are capped to fit this budget")
    ap.add_argument("--stream-count", type=int, default=20000)
    ap.add_argument("--no-stream", action="store_true", help="skip the batching / serving stream")
    ap.add_argument("--host-staging-gib", type=int, default=8,
                    help="page-locked host staging of the batch engine (stream)")
    ap.add_argument("--arena-gib", type=int, default=16)
    ap.add_argument("--chunk-sweeps", type=int, default=16)
    ap.add_argument("--no-serve-tune", action="store_true",
                    help="stream: skip the batch engine's knob tuning on the first graphs")
    ap.add_argument("--serve-tune-graphs", type=int, default=2000)
    ap.add_argument("--check-workers", type=int, default=12,
                    help="oracle processes that check every stream result")
    ap.add_argument("--autotune", dest="autotune", action="store_true", default=None,
                    help="tune the sweep knobs on the workload first (default for rmat24_planted)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--graph", dest="graph", action="store_true", default=None,
                    help="runs replay a captured CUDA graph (KCORE_GRAPH; default for rmat24_planted)")
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--options", default=None,
                    help='kcore_options fields as JSON (e.g. \'{"relabel": 2, "block": 256}\'); '
                         'replaces the autotuner')
    a = ap.parse_args()
    heavy = a.workload == "rmat24_planted"
    if a.autotune is None:
        a.autotune = heavy and a.options is None
    if a.graph is None:
        a.graph = heavy
    return a


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock, max clock and throttle reasons sampled every millisecond
    during the timed region through NVML (read-only queries via ctypes), or
    every 100 ms through nvidia-smi when NVML cannot be loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.bus = None
        try:
            import torch
            p = torch.cuda.get_device_properties(index)
            self.bus = f"{getattr(p, 'pci_domain_id', 0):08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
        except Exception:
            pass
        self.index = index
        self.samples = []      # (sm_mhz, max_mhz, reason bits)
        self._stop = threading.Event()
        self._t = None
        self._nvml = self._open_nvml()

    def _open_nvml(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            ok = -1
            if self.bus:
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(self.bus.encode(), ctypes.byref(h))
            if ok != 0:
                ok = lib.nvmlDeviceGetHandleByIndex_v2(self.index, ctypes.byref(h))
            if ok != 0:
                return None
            reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            return lib, h, reasons
        except Exception:
            return None

    def _sample_nvml(self):
        import ctypes
        lib, h, reasons = self._nvml
        c, m, r = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(c))
        lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(m))
        reasons(h, ctypes.byref(r))
        self.samples.append((float(c.value), float(m.value), int(r.value)))

    def _sample_smi(self):
        out = subprocess.run(["nvidia-smi", f"--id={self.bus or self.index}", f"--query-gpu={self.Q}",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=5).stdout.strip()
        f = [x.strip() for x in out.split(",")]
        if len(f) >= 6 and f[0].replace(".", "").isdigit():
            bits = sum(b for b, v in zip((0x8, 0x40, 0x20, 0x4), f[2:6]) if v.lower() == "active")
            self.samples.append((float(f[0]), float(f[1]), bits))

    def _run(self):
        period = 0.001 if self._nvml else 0.1
        while not self._stop.is_set():
            try:
                self._sample_nvml() if self._nvml else self._sample_smi()
            except Exception:
                pass
            self._stop.wait(period)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)
        if not self.samples:          # a region shorter than one sample: take one now
            try:
                self._sample_nvml() if self._nvml else self._sample_smi()
            except Exception:
                pass

    def summary(self):
        sm = [x[0] for x in self.samples]
        mx = [x[1] for x in self.samples]
        bits = 0
        for x in self.samples:
            bits |= x[2]
        reasons = sorted(name for b, name in self.REASONS.items() if bits & b)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples), "source": "nvml" if self._nvml else "nvidia-smi"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sweep_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("sweep.cu", "kc_common.cuh"):
        with open(os.path.join(ROOT, "paper_2512_00233_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per sweep-kernel launch from the committed ncu summary, or
    None when the kernel source changed since the capture."""
    try:
        with open(PROFILE_TRAFFIC) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("source_hash") == sweep_source_hash():
            return int(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# ---------------------------------------------------------------- ranks
def combine_ranks(local_ms: float, units_per_rank: float, steps: int, device=None):
    """Whole-job figures over the ranks of the default process group (or this
    process alone): the time is the maximum over ranks, the units the sum of
    every rank's.  Returns (max_ms, units_per_second)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = local_ms
    if ws > 1:
        x = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, units_per_rank * steps * ws / (t / 1e3)


# ---------------------------------------------------------------- oracle on the host
def oracle_peel_baseline(workload: str, budget_s: float, omp_threads: int = 4) -> dict:
    """The oracle on the whole workload, in a process of its own: its host CSR
    build, then Batagelj-Zaversnik peels (single thread), each timed; as many
    peels (1..5) as fit the budget after the first.  Generation of the samples
    (OpenMP, `omp_threads`) is not timed."""
    os.environ["OMP_NUM_THREADS"] = str(omp_threads)   # before graphgen's library loads
    import graphgen
    import oracle
    g = graphgen.workload(workload)
    n, samples = g.n, g.samples
    t0 = time.perf_counter()
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    csr_s = time.perf_counter() - t0
    del g
    peels = []
    while True:
        t0 = time.perf_counter()
        core = oracle.coreness(n, rp, col)
        peels.append(time.perf_counter() - t0)
        if len(peels) >= 5 or sum(peels) + peels[0] > budget_s:
            break
    return {"n": n, "samples": samples, "m": int(rp[-1]) // 2, "csr_s": csr_s, "peels": peels,
            "kmax": int(core.max()) if n else 0}


def cpu_baseline_line(r: dict) -> dict:
    mean = statistics.mean(r["peels"])
    return {"value": r["m"] / mean, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"whole workload (n {r['n']}, m {r['m']}): {len(r['peels'])} "
                      f"Batagelj-Zaversnik peel(s) of the oracle's own host CSR, single thread, "
                      f"mean {mean:.3f} s; the oracle's host CSR build took {r['csr_s']:.1f} s "
                      f"(reported apart, not in the value)",
            "peel_s": r["peels"], "csr_build_s": r["csr_s"]}


def run_reference(args):
    """The oracle as it stands on the host cores: the whole workload's host CSR
    built once (timed, reported apart), then timed peels.  One peel of the
    largest workload takes tens of seconds, so the timed peels are capped to
    fit --ref-budget-s (at least one); the line states the count."""
    import graphgen
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    g = graphgen.workload(args.workload)
    name, n, samples = g.name, g.n, g.samples
    t0 = time.perf_counter()
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    csr_s = time.perf_counter() - t0
    del g
    m = int(rp[-1]) // 2
    warm = min(args.warmup, 1)
    t_est = None
    for _ in range(warm):
        t0 = time.perf_counter()
        oracle.coreness(n, rp, col)
        t_est = time.perf_counter() - t0
    times = []
    while len(times) < args.steps:
        t0 = time.perf_counter()
        oracle.coreness(n, rp, col)
        times.append(time.perf_counter() - t0)
        t_est = t_est or times[0]
        if len(times) >= max(1, int(args.ref_budget_s // t_est)):
            break
    total = sum(times)
    value = m * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": len(times), "steps_requested": args.steps, "warmup": warm,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(name, n, samples, m),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"whole workload; {len(times)} timed Batagelj-Zaversnik peel(s) "
                                   f"of the oracle's own host CSR (built once in {csr_s:.1f} s, "
                                   f"not timed), single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "csr_build_s": csr_s,
    }
    print(json.dumps(line), flush=True)


def workload_config(name, n, samples, m) -> dict:
    """The `config` object, the same for both arms."""
    return {"workload": name, "n": n, "samples": samples, "m": m,
            "l2": "512 MiB buffer rewritten between timed steps"}


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch

    import graphgen
    import paper_2512_00233_gb300 as K

    ws, rank, local = dist_env()
    # the oracle's CPU baseline runs in a spawned process of its own once the
    # timed GPU work is over (its host CSR build would compete with the host
    # copies of the timed regions), beside the stream's result check
    cpu = {}

    def start_cpu_baseline():
        if ws == 1 and not args.no_cpu_baseline and not cpu:
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            cpu["pool"] = ProcessPoolExecutor(1, mp_context=mp.get_context("spawn"))
            cpu["job"] = cpu["pool"].submit(oracle_peel_baseline, args.workload, args.cpu_budget_s)

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    g0 = graphgen.workload(args.workload)
    rp_bytes = g0.meta["row_ptr_bytes"]
    src_d = torch.from_numpy(g0.src).to(dev)
    dst_d = torch.from_numpy(g0.dst).to(dev)
    out_d = torch.empty(g0.n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def flush_l2():
        flush.add_(1)

    opts = None
    tuned = None
    t_tune = 0.0
    if args.options:
        tuned = json.loads(args.options)
        opts = K.default_options(**tuned)
    elif args.autotune:
        # the vertex numbering first (fixed when a graph is made), then the
        # sweep knobs on a graph with that numbering
        from paper_2512_00233_gb300 import autotune
        t0 = time.perf_counter()
        order, order_ms = autotune.pick_order(
            lambda r: K.Graph.from_coo(g0.n, src_d, dst_d, rp_bytes, options=K.default_options(relabel=r)),
            reps=2)
        with K.Graph.from_coo(g0.n, src_d, dst_d, rp_bytes, options=K.default_options(relabel=order)) as gt:
            opts, _ = autotune.autotune(gt, reps=2, passes=1, cache=None)
        opts.relabel = order
        t_tune = time.perf_counter() - t0
        tuned = {k: getattr(opts, k) for k in autotune.SPACE}
        tuned["relabel"] = order
        tuned["relabel_sweep_ms"] = {str(k): v for k, v in order_ms.items()}

    def step_device():
        g = K.Graph.from_coo(g0.n, src_d, dst_d, rp_bytes, options=opts)
        g.run(out=out_d, graph=args.graph)
        return g

    # warm-up (also gives m and the per-run statistics)
    for _ in range(args.warmup):
        flush_l2()
        step_device().close()
    torch.cuda.synchronize()

    # ---- timed region: K whole steps, device-resident inputs
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    launches0 = K.lib().kcore_kernel_launches()
    with ClockSampler(dev) as clocks:
        barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush_l2()
            ev[i][0].record(stream)
            g = step_device()
            ev[i][1].record(stream)
            stats.append(g.stats())      # waits for the step; outside the event pair
            g.close()
        torch.cuda.synchronize()
        barrier()
        t_wall = time.perf_counter() - t_wall
    launches = (K.lib().kcore_kernel_launches() - launches0) / args.steps
    step_ms = [a.elapsed_time(b) for a, b in ev]
    m = stats[0]["nnz"] // 2
    local_ms, value = combine_ranks(sum(step_ms), m, args.steps, device=dev)

    # ---- decomposition alone on the resident graph (paper's timing)
    g = K.Graph.from_coo(g0.n, src_d, dst_d, rp_bytes, options=opts)
    run_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    sweep_stats = []
    for _ in range(2):
        flush_l2()
        g.run(out=out_d, graph=args.graph)
    for i in range(args.steps):
        flush_l2()
        run_ev[i][0].record(stream)
        g.run(out=out_d, graph=args.graph)
        run_ev[i][1].record(stream)
        sweep_stats.append(g.stats())
    torch.cuda.synchronize()
    run_ms = [a.elapsed_time(b) for a, b in run_ev]
    g.close()

    # ---- end to end through the C ABI with host buffers
    src_h = torch.from_numpy(g0.src).pin_memory()
    dst_h = torch.from_numpy(g0.dst).pin_memory()
    out_h = torch.empty(g0.n, dtype=torch.int32).pin_memory()
    e2e_t, e2e_create, e2e_run, e2e_call = [], [], [], []
    for i in range(args.warmup + args.steps):
        flush_l2()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gh = K.Graph.from_coo(g0.n, src_h.numpy(), dst_h.numpy(), rp_bytes, options=opts)
        tc = time.perf_counter()
        gh.run(out=out_h.numpy())
        t1 = time.perf_counter()
        st_h = gh.stats()
        gh.close()
        if i >= args.warmup:
            e2e_t.append(t1 - t0)
            e2e_call.append(tc - t0)
            e2e_create.append(st_h["ms_create"])
            e2e_run.append(st_h["ms_run"])
    e2e_value = m * ws / statistics.mean(e2e_t)
    del src_h, dst_h, src_d, dst_d

    # ---- roofline of the sweep kernel (dominant kernel of the decomposition)
    peak, peak_kind = measured_peaks()
    bytes_alg = statistics.mean(s["bytes_algorithmic"] for s in sweep_stats)
    sweep_ms = statistics.mean(s["ms_sweep"] for s in sweep_stats)
    achieved = bytes_alg / (sweep_ms / 1e3) / 1e9
    traffic = profiled_traffic(args.workload)

    line = None
    if rank == 0:
        create_ms = statistics.mean(s["ms_create"] for s in stats)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": local_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": workload_config(g0.name, g0.n, g0.samples, m),
            "setup": {"row_ptr_bytes": rp_bytes,
                      "step": "kcore_create_coo (device samples) + kcore_run (device output"
                              + (", replayed CUDA graph)" if args.graph else ")"),
                      "inputs_vs_l2": f"{8 * g0.samples / 2**30:.2f} GiB of samples against a "
                                      "129 MB L2",
                      "options": tuned or "library defaults",
                      "autotune_s": t_tune},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * g0.samples,
                    "d2h_bytes_per_step": 4 * g0.n,
                    "ms_per_step": 1e3 * statistics.mean(e2e_t),
                    "create_call_ms": 1e3 * statistics.mean(e2e_call),
                    "create_events_ms": statistics.mean(e2e_create),
                    "run_events_ms": statistics.mean(e2e_run)},
            "gpu_launches": launches,
            "create_ms": create_ms,
            "decompose": {"value": m / (statistics.mean(run_ms) / 1e3), "unit": UNIT,
                          "ms_run": statistics.mean(run_ms), "ms_sweep": sweep_ms,
                          "sweeps": statistics.mean(s["sweeps"] for s in sweep_stats),
                          "tail_sweeps": statistics.mean(s["tail_sweeps"] for s in sweep_stats),
                          "evaluated": statistics.mean(s["evaluated"] for s in sweep_stats),
                          "edges_scanned": statistics.mean(s["edges_scanned"] for s in sweep_stats),
                          "grid": sweep_stats[0]["grid"], "block": sweep_stats[0]["block"],
                          "cuda_graph": bool(args.graph)},
            "roofline": {"kernel": "k_sweep", "bound": "hbm", "achieved": achieved, "peak": peak,
                         "peak_kind": f"{peak_kind} HBM copy GB/s", "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "bytes_per_launch": bytes_alg},
            "clocks": clocks.summary(),
            "wall_s": t_wall,
        }
    del g0
    if rank == 0 and ws == 1 and not args.no_stream:
        line["stream"] = run_stream(args, K, torch, after_timed=start_cpu_baseline)
    start_cpu_baseline()
    if line is not None and cpu:
        line["cpu_baseline"] = cpu_baseline_line(cpu["job"].result())
        cpu["pool"].shutdown()
    if line is not None:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched / served stream
def result_hash(core) -> bytes:
    import numpy as np
    return hashlib.blake2b(np.ascontiguousarray(core, dtype=np.int32).tobytes(),
                           digest_size=16).digest()


def oracle_stream_hashes(lo: int, hi: int) -> list:
    """Oracle coreness hashes of stream graphs [lo, hi) (a spawned worker)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import graphgen
    import oracle
    out = []
    for i in range(lo, hi):
        g = graphgen.stream_graph(i)
        rp, col = oracle.csr_build(g.n, g.src, g.dst)
        out.append((i, result_hash(oracle.coreness(g.n, rp, col)), int(rp[-1]) // 2))
    return out


def percentiles_ms(lat_s):
    import numpy as np
    a = np.asarray(lat_s) * 1e3
    return float(np.percentile(a, 50)), float(np.percentile(a, 99))


def serve_one_launch(K, graphs, arrivals):
    """One kcore_create_coo + kcore_run (host samples in, host coreness out) per
    request, by one server thread in arrival order.  `arrivals` None: every
    request at once.  Latency = result in the caller's buffer - arrival
    (time.perf_counter, CLOCK_MONOTONIC)."""
    import queue

    import numpy as np
    G = len(graphs)
    lat = np.zeros(G)
    res = [None] * G
    q = queue.SimpleQueue()

    def server():
        while True:
            item = q.get()
            if item is None:
                return
            i, t_arr = item
            g = graphs[i]
            with K.Graph.from_coo(g.n, g.src, g.dst) as gg:
                res[i] = gg.run(device=False)
            lat[i] = time.perf_counter() - t_arr

    th = threading.Thread(target=server, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for i in range(G):
        if arrivals is not None:
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
        q.put((i, time.perf_counter()))
    q.put(None)
    th.join()
    return time.perf_counter() - t0, lat, res


def serve_batched(K, opts, graphs, arrivals):
    """The continuous-batching engine under the same arrivals: requests are
    submitted at their arrival times while a poller thread collects results.
    Latency = the engine's result-ready time (kcore_poll_info done_s, the same
    monotonic clock) - arrival."""
    import queue

    import numpy as np
    G = len(graphs)
    t_arr = np.zeros(G)
    lat = np.zeros(G)
    res = [None] * G
    infos = [None] * G
    q = queue.SimpleQueue()
    clock_ok = [True]
    errors = []
    with K.BatchEngine(opts) as eng:
        for g in graphs[:3]:                       # warm-up
            eng.poll(eng.submit_coo(g.n, g.src, g.dst), g.n, timeout_us=-1)

        def poller():
            while True:
                item = q.get()
                if item is None:
                    return
                i, t = item
                st, core, info = eng.poll_info(t, graphs[i].n, timeout_us=-1)
                if st != K.KCORE_OK:
                    errors.append(f"stream graph {i}: status {st}")
                    continue
                res[i], infos[i] = core, info
                lat[i] = info["done_s"] - t_arr[i]
                if not (t_arr[i] <= info["submit_s"] <= info["done_s"]):
                    clock_ok[0] = False

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for i in range(G):
            if arrivals is not None:
                delay = t0 + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            g = graphs[i]
            t_arr[i] = time.perf_counter()
            q.put((i, eng.submit_coo(g.n, g.src, g.dst)))
        q.put(None)
        th.join()
        wall = time.perf_counter() - t0
        stats = eng.stats()
    if errors:
        raise RuntimeError("; ".join(errors[:5]))
    if not clock_ok[0]:
        raise RuntimeError("engine times are not on the clock of time.perf_counter")
    overlap = sum(1 for x in infos if x["resident_at_admit"] > 0)
    return wall, lat, res, stats, overlap


def autotune_serve_space():
    from paper_2512_00233_gb300 import autotune
    return list(autotune.SERVE_SPACE)


def run_stream(args, K, torch, after_timed=None):
    """The batching / serving workload: the first --stream-count graphs of the
    stream (n log-uniform in [100, 200000]; ER avg degree 8, R-MAT 8n samples,
    damaged grid), host samples.  Both servers run for real, one after the
    other on this GPU: saturated (every request at once) and under Poisson
    arrivals at 0.7 x each server's saturated rate; every result of every run
    is compared with the oracle's coreness afterwards (spawned processes)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor, ThreadPoolExecutor

    import graphgen
    G = args.stream_count
    graphgen.stream_params(0)                        # loads the generator before the threads
    t0 = time.perf_counter()
    with ThreadPoolExecutor(min(16, os.cpu_count() or 4)) as ex:
        graphs = list(ex.map(graphgen.stream_graph, range(G)))
    t_gen = time.perf_counter() - t0
    opts = K.default_serve_options(mem_budget=args.arena_gib << 30, chunk_sweeps=args.chunk_sweeps,
                                   host_staging=args.host_staging_gib << 30)
    serve_tuned, t_tune = None, 0.0
    if not args.no_serve_tune:
        # the engine's knobs tuned on the first graphs of the stream (saturated
        # graphs/s; every candidate's results checked against the first's)
        import copy

        from paper_2512_00233_gb300 import autotune
        t0 = time.perf_counter()
        base = copy.copy(opts)
        base.host_staging = min(opts.host_staging, 2 << 30)
        best, _ = autotune.autotune_serve(graphs[:min(G, args.serve_tune_graphs)], base, reps=1)
        opts.chunk_sweeps = best.chunk_sweeps
        opts.sweep = best.sweep
        t_tune = time.perf_counter() - t0
        serve_tuned = {"chunk_sweeps": best.chunk_sweeps,
                       **{k: getattr(best.sweep, k) for k in autotune.SERVE_SPACE if k != "chunk_sweeps"}}
    serve_one_launch(K, graphs[:3], None)            # warm-up
    runs = {}
    hashes = {}

    def keep(name, res):
        hashes[name] = [result_hash(r) for r in res]

    with ClockSampler(torch.cuda.current_device()) as clocks:
        wall, lat, res = serve_one_launch(K, graphs, None)
        runs["one_launch_saturated"] = {"graphs_per_s": G / wall, "wall_s": wall}
        keep("one_launch_saturated", res)
        cap1 = G / wall
        wall, lat, res, st, ov = serve_batched(K, opts, graphs, None)
        runs["batched_saturated"] = {"graphs_per_s": G / wall, "wall_s": wall,
                                     "launches": st["launches"], "admissions": st["admissions"],
                                     "admitted_while_busy": st["admitted_while_busy"],
                                     "busy_s": st["busy_s"], "admit_s": st["admit_s"],
                                     "sweep_s": st["sweep_s"], "retire_s": st["retire_s"]}
        keep("batched_saturated", res)
        cap2 = G / wall
        for tag, rate, seed in (("at_0.7x_one_launch", 0.7 * cap1, 1),
                                ("at_0.7x_batched", 0.7 * cap2, 2)):
            arr = graphgen.poisson_arrivals(G, rate, seed=seed)
            wall, lat, res = serve_one_launch(K, graphs, arr)
            p50, p99 = percentiles_ms(lat)
            runs[f"one_launch_{tag}"] = {"arrival_rate_per_s": rate, "graphs_per_s": G / wall,
                                         "p50_ms": p50, "p99_ms": p99}
            keep(f"one_launch_{tag}", res)
            wall, lat, res, st, ov = serve_batched(K, opts, graphs, arr)
            p50, p99 = percentiles_ms(lat)
            runs[f"batched_{tag}"] = {"arrival_rate_per_s": rate, "graphs_per_s": G / wall,
                                      "p50_ms": p50, "p99_ms": p99, "launches": st["launches"],
                                      "admitted_while_busy": st["admitted_while_busy"],
                                      "admitted_into_busy_arena": ov}
            keep(f"batched_{tag}", res)
    del res, graphs
    if after_timed is not None:
        after_timed()
    # every result against the oracle (outside the timed runs)
    t0 = time.perf_counter()
    workers = max(1, min(args.check_workers, os.cpu_count() or 1))
    step = max(1, G // (workers * 8))
    expect, m_total = [None] * G, 0
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        for part in ex.map(oracle_stream_hashes, range(0, G, step),
                           [min(G, lo + step) for lo in range(0, G, step)]):
            for i, h, m in part:
                expect[i] = h
                m_total += m
    t_check = time.perf_counter() - t0
    bad = {name: [i for i in range(G) if hs[i] != expect[i]] for name, hs in hashes.items()}
    mismatches = {k: v[:10] for k, v in bad.items() if v}
    if mismatches:
        raise RuntimeError(f"stream results differ from the oracle: {mismatches}")
    return {
        "workload": "graph stream (first %d graphs; n log-uniform in [100, 200000]; "
                    "ER avg degree 8 / R-MAT 8n samples / damaged grid)" % G,
        "graphs": G, "m_total": m_total, "metric": "graphs/s and p50/p99 latency",
        "arena_gib": args.arena_gib, "host_staging_gib": args.host_staging_gib,
        "chunk_sweeps": opts.chunk_sweeps,
        "serve_options": serve_tuned or "library defaults",
        "serve_tune": (f"coordinate descent over {sorted(autotune_serve_space())} "
                       f"on the first {min(G, args.serve_tune_graphs)} graphs, {t_tune:.1f} s")
        if serve_tuned else None,
        "latency": "arrival (time.perf_counter before the request is handed in) to the result "
                   "on the host; one launch per graph: coreness in the caller's buffer; batched: "
                   "the engine's result-ready time on the same monotonic clock",
        "runs": runs,
        "batched_edges_per_s": m_total / runs["batched_saturated"]["wall_s"],
        "results_checked": G * len(hashes), "graphs_checked": G, "check": "oracle coreness, "
        "blake2b-128 of every result, all runs", "generate_s": t_gen, "check_s": t_check,
        "clocks": clocks.summary(),
    }


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "stream":
        import torch

        import paper_2512_00233_gb300 as K
        torch.cuda.set_device(0)
        s = run_stream(args, K, torch)
        r = s["runs"]["batched_saturated"]
        line = {"metric": "batched graphs/s", "value": r["graphs_per_s"], "unit": "graphs/s",
                "n_gpus": 1, "steps": 1, "warmup": 3, "ms_per_step": 1e3 * r["wall_s"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic", "config": {"workload": s["workload"]},
                "stream": s}
        print(json.dumps(line), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
