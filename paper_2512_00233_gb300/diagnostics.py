"""Convergence diagnostics of a run (the quantities of Fig. 4 and Fig. 5).

Per sweep s of the last run of a graph:

* ``activated`` -- vertices evaluated in sweep s, and ``pct_activated`` =
  activated / n * 100 (Fig. 5);
* ``mean_error`` -- mean over all vertices of |est_v - core_v| after sweep s
  (Fig. 4).  Estimates start at the degree and never go below the coreness
  (the h-operator is monotone and the coreness is its largest fixed point,
  Sec. III), so |est_v - core_v| = est_v - core_v and
      sum_v |est_v - core_v| = sum_v deg_v - sum_{s' <= s} decrease[s'] - sum_v core_v,
  where decrease[s'] is the sum of the estimate decreases made in sweep s'
  (recorded on the device).  No estimates are copied out per sweep.

``convergence(graph)`` returns the rows; ``write_csv(rows, path)`` writes them.
"""
from __future__ import annotations

import csv

import numpy as np

from . import Graph

COLUMNS = ("sweep", "activated", "pct_activated", "degree_sum", "entries_read", "updates",
           "decrease", "mean_error", "start_us")


def convergence(graph: Graph, coreness=None) -> list[dict]:
    """Rows of the last run of `graph`.  `coreness`: the run's result (host
    array or CUDA tensor); copied from a fresh run when None."""
    n = graph.n
    if coreness is None:
        coreness = graph.run(device=False)
    core = coreness.cpu().numpy() if hasattr(coreness, "cpu") else np.asarray(coreness)
    f, dsum, upd, t = graph.trace(with_time=True)
    read, dec = graph.trace_detail()
    deg_sum = int(np.diff(graph.row_ptr_host().astype(np.int64)).sum())
    core_sum = int(core.astype(np.int64).sum())
    excess = deg_sum - core_sum - np.cumsum(dec)
    rows = []
    for s in range(len(f)):
        rows.append({
            "sweep": s,
            "activated": int(f[s]),
            "pct_activated": 100.0 * int(f[s]) / max(n, 1),
            "degree_sum": int(dsum[s]),
            "entries_read": int(read[s]),
            "updates": int(upd[s]),
            "decrease": int(dec[s]),
            "mean_error": float(excess[s]) / max(n, 1),
            "start_us": float(t[s]) / 1e3,
        })
    return rows


def write_csv(rows: list[dict], path: str) -> None:
    with open(path, "w", newline="") as fh:
        w = csv.DictWriter(fh, fieldnames=COLUMNS)
        w.writeheader()
        for r in rows:
            w.writerow(r)
