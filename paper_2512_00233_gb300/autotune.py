"""Autotuner of the sweep engine's launch knobs.

Coordinate descent over the degree-tier thresholds (t_lo, t_hi), the CTA
size, the work-grab sizes and the single-CTA tail threshold: each knob in
turn is set to each of its candidate values with the others fixed, the graph
is decomposed a few times, and the value with the lowest median sweep-kernel
time
(CUDA events recorded by the library around the launch) is kept.  Two passes.
Every candidate run is checked to give the same coreness as the first.

Results are cached in a JSON file keyed by coarse degree statistics (log2 of
n, of the average degree and of the maximum degree), so graphs of the same
shape reuse a tuning: `tuned_options(graph)`.

`autotune_serve` tunes the batch engine the same way on a sample of a graph
stream: sweeps per persistent launch, the sweep knobs of the arena and the
cleaner its admissions use, by the saturated throughput (graphs/s) of the
sample, every result checked against the first candidate's.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import numpy as np

from . import Graph, Options, default_options

SPACE = {
    "t_lo": [4, 8, 16],
    "t_hi": [64, 256, 512, 1024, 2048],
    "block": [256, 512],
    "low_chunk": [2, 4, 8],
    "med_chunk": [1, 4, 16],
    "tail_max": [256, 1024, 4096],
}

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "kcore_gb300", "autotune.json")


def shape_key(graph: Graph) -> str:
    rp = graph.row_ptr_host()
    deg = np.diff(rp.astype(np.int64))
    n = max(graph.n, 1)
    avg = max(graph.nnz / n, 1e-9)
    mx = int(deg.max()) if deg.size else 0
    return f"n{round(math.log2(n))}_avg{round(math.log2(avg + 1))}_max{round(math.log2(mx + 1))}"


def _time(graph: Graph, opts: Options, reps: int, check=None) -> float:
    graph.set_options(opts)
    times = []
    out = None
    for _ in range(reps + 1):
        out = graph.run()
        times.append(graph.stats()["ms_sweep"])
    if check is not None:
        assert bool((out == check).all()), "autotune candidate changed the result"
    return statistics.median(times[1:])


def autotune(graph: Graph, reps: int = 3, passes: int = 2, space: dict | None = None,
             cache: str | None = DEFAULT_CACHE, verbose: bool = False):
    """Returns (best Options, list of (knob, value, ms) trials) and records the
    result in `cache` (None: no file)."""
    space = space or SPACE
    d = default_options()
    best = {k: getattr(d, k) for k in space}
    ref = graph.run()
    best_ms = _time(graph, default_options(**best), reps, ref)
    trials = [("default", None, best_ms)]
    for _ in range(passes):
        for knob, values in space.items():
            for val in values:
                if val == best[knob]:
                    continue
                cand = dict(best, **{knob: val})
                if cand.get("t_hi", d.t_hi) < cand.get("t_lo", d.t_lo):
                    continue
                ms = _time(graph, default_options(**cand), reps, ref)
                trials.append((knob, val, ms))
                if verbose:
                    print(f"autotune {knob}={val}: {ms:.3f} ms (best {best_ms:.3f})")
                if ms < best_ms:
                    best, best_ms = cand, ms
    opts = default_options(**best)
    graph.set_options(opts)
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        data = {}
        if os.path.exists(cache):
            with open(cache) as f:
                data = json.load(f)
        data[shape_key(graph)] = {"options": best, "ms_sweep": best_ms}
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return opts, trials


def pick_order(make_graph, reps: int = 3, orders=(1, 2, -1)):
    """The vertex numbering (kcore_options.relabel, fixed when a graph is made)
    with the lowest median sweep time: make_graph(relabel) builds the graph.
    Every candidate is checked to give the same coreness.  Returns (relabel,
    {relabel: ms})."""
    times, ref = {}, None
    for r in orders:
        with make_graph(r) as g:
            out = g.run()
            if ref is None:
                ref = out.cpu()
            assert bool((out.cpu() == ref).all()), "numbering changed the result"
            ms = []
            for _ in range(reps):
                g.run(out=out)
                ms.append(g.stats()["ms_sweep"])
            times[r] = statistics.median(ms)
    best = min(times, key=times.get)
    return best, times


def tuned_options(graph: Graph, cache: str = DEFAULT_CACHE) -> Options | None:
    """Cached tuning for graphs of this shape, or None."""
    if not os.path.exists(cache):
        return None
    with open(cache) as f:
        data = json.load(f)
    e = data.get(shape_key(graph))
    return default_options(**e["options"]) if e else None


SERVE_SPACE = {
    "chunk_sweeps": [4, 8, 16, 32, 64],
    "block": [256, 512],
    "t_hi": [256, 1024, 2048],
    "med_chunk": [1, 4, 16],
    "build_sort": [0, 1, -1],   # the admission's cleaner: automatic, sorted, counted
}


def _serve_rate(graphs, opts, reps: int, check=None):
    """Median saturated graphs/s of the batch engine on `graphs` (every one
    submitted at once, then polled), and the results of the last repetition."""
    import time

    from . import BatchEngine
    rates, res = [], None
    for _ in range(reps):
        with BatchEngine(opts) as eng:
            t0 = time.perf_counter()
            tickets = [eng.submit_coo(g.n, g.src, g.dst) for g in graphs]
            res = [eng.poll(t, g.n, timeout_us=-1)[1] for g, t in zip(graphs, tickets)]
            rates.append(len(graphs) / (time.perf_counter() - t0))
    if check is not None:
        for a, b in zip(res, check):
            assert a is not None and np.array_equal(a, b), "serve candidate changed a result"
    return statistics.median(rates), res


def autotune_serve(graphs, base, reps: int = 2, passes: int = 1, space: dict | None = None,
                   verbose: bool = False):
    """Coordinate descent over SERVE_SPACE for the batch engine on a stream
    sample.  `base`: a ServeOptions to start from (mem_budget, staging, ...).
    Returns (best ServeOptions, trials [(knob, value, graphs/s)])."""
    import copy

    space = space or SERVE_SPACE

    def make(knobs):
        o = copy.copy(base)
        sw = copy.copy(base.sweep)
        for k, v in knobs.items():
            if k == "chunk_sweeps":
                o.chunk_sweeps = v
            else:
                setattr(sw, k, v)
        o.sweep = sw
        return o

    best = {"chunk_sweeps": base.chunk_sweeps}
    best.update({k: getattr(base.sweep, k) for k in space if k != "chunk_sweeps"})
    best_rate, ref = _serve_rate(graphs, make(best), reps)
    trials = [("base", None, best_rate)]
    for _ in range(passes):
        for knob, values in space.items():
            for val in values:
                if val == best[knob]:
                    continue
                cand = dict(best, **{knob: val})
                if cand.get("t_hi", 2048) < base.sweep.t_lo:
                    continue
                rate, _ = _serve_rate(graphs, make(cand), reps, ref)
                trials.append((knob, val, rate))
                if verbose:
                    print(f"autotune_serve {knob}={val}: {rate:.0f} graphs/s (best {best_rate:.0f})")
                if rate > best_rate:
                    best, best_rate = cand, rate
    return make(best), trials
