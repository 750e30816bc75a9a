"""Host-side logic that needs no GPU, driven by fake graph objects with the
methods of `paper_2512_00233_gb300.Graph` that it uses:

- the autotuner's coordinate descent (it finds the optimum of a separable cost,
  never times a candidate with t_hi < t_lo, refuses a candidate that changes
  the result, and caches by graph shape);
- the convergence diagnostics' arithmetic (Fig. 4 / Fig. 5 quantities): given a
  per-sweep trace consistent with synchronous rounds of the oracle, the mean
  error per sweep equals the oracle's mean |est - core| after that round.

The option defaults come from the library's host-only kcore_default_options.
"""
import csv

import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K
from paper_2512_00233_gb300 import autotune, diagnostics

BEST = {"t_lo": 8, "t_hi": 1024, "block": 256, "low_chunk": 4, "med_chunk": 16, "tail_max": 256}


def separable_cost(o):
    """Sweep time with a unique minimum at BEST, each knob contributing alone."""
    ms = 1.0
    for k, v in BEST.items():
        ms += 0.1 * abs(np.log2(getattr(o, k)) - np.log2(v))
    return ms


class FakeGraph:
    def __init__(self, cost, n=1000, max_deg=40, changes_with=None):
        self.cost, self.n, self.changes_with = cost, n, changes_with
        self.opts = K.default_options()
        deg = np.full(n, 4, np.int64)
        deg[0] = max_deg
        self.rp = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
        self.nnz = int(self.rp[-1])
        self.timed = []

    def set_options(self, o):
        self.opts = o

    def run(self, **kw):
        out = np.arange(self.n) % 5
        if self.changes_with and all(getattr(self.opts, k) == v for k, v in self.changes_with.items()):
            out = out + 1
        return out

    def stats(self):
        self.timed.append({k: getattr(self.opts, k) for k in BEST})
        return {"ms_sweep": self.cost(self.opts)}

    def row_ptr_host(self):
        return self.rp


def test_autotune_finds_separable_optimum_and_caches(tmp_path):
    g = FakeGraph(separable_cost)
    cache = str(tmp_path / "tune.json")
    opts, trials = autotune.autotune(g, reps=1, passes=2, cache=cache)
    assert {k: getattr(opts, k) for k in BEST} == BEST
    assert trials[0][0] == "default" and min(t[2] for t in trials) == pytest.approx(1.0)
    assert {k: getattr(g.opts, k) for k in BEST} == BEST        # left applied to the graph
    got = autotune.tuned_options(g, cache)
    assert got is not None and {k: getattr(got, k) for k in BEST} == BEST
    other = FakeGraph(separable_cost, n=1 << 16, max_deg=5000)  # another shape: no entry
    assert autotune.shape_key(other) != autotune.shape_key(g)
    assert autotune.tuned_options(other, cache) is None


def test_autotune_skips_t_hi_below_t_lo():
    g = FakeGraph(lambda o: 1.0 + 0.01 * o.t_hi)
    space = {"t_lo": [16], "t_hi": [8, 64, 2048]}
    opts, trials = autotune.autotune(g, reps=1, passes=1, space=space, cache=None)
    assert all(t["t_hi"] >= t["t_lo"] for t in g.timed)
    assert not any(t[0] == "t_hi" and t[1] == 8 for t in trials)
    assert opts.t_hi == 64


def test_autotune_refuses_a_candidate_that_changes_the_result():
    g = FakeGraph(separable_cost, changes_with={"block": 256})
    with pytest.raises(AssertionError):
        autotune.autotune(g, reps=1, passes=1, cache=None)


class TraceGraph:
    """A graph whose per-sweep trace is that of the oracle's synchronous rounds."""

    def __init__(self, n, rp, col, refined):
        self.n = n
        self.rp = rp
        rounds, _, fr, _ = oracle.montresor_sync(n, rp, col, refined=refined, record=1 << 20)
        deg = np.diff(rp.astype(np.int64))
        prev = deg.copy()
        self.f, self.dec, self.est = fr, [], []
        for s in range(rounds):
            _, est, _, _ = oracle.montresor_sync(n, rp, col, max_rounds=s + 1, refined=refined)
            est = est.astype(np.int64)
            self.dec.append(int((prev - est).sum()))
            self.est.append(est)
            prev = est
        self.dec = np.array(self.dec, np.int64)

    def trace(self, with_time=False):
        k = len(self.f)
        z = np.zeros(k, np.int64)
        return (self.f, z, z, np.arange(k, dtype=np.int64) * 1000) if with_time else (self.f, z, z)

    def trace_detail(self):
        return np.zeros(len(self.f), np.int64), self.dec

    def row_ptr_host(self):
        return self.rp


@pytest.mark.parametrize("refined", [False, True])
def test_diagnostics_mean_error_follows_the_rounds(tmp_path, refined):
    g0 = graphgen.damaged_grid(48, seed=4)
    rp, col = oracle.csr_build(g0.n, g0.src, g0.dst)
    core = oracle.coreness(g0.n, rp, col)
    tg = TraceGraph(g0.n, rp, col, refined)
    rows = diagnostics.convergence(tg, core)
    assert len(rows) == len(tg.est) > 1
    for s, r in enumerate(rows):
        expect = float((tg.est[s] - core).sum()) / g0.n
        assert r["mean_error"] == pytest.approx(expect, abs=0.0)
        assert r["pct_activated"] == pytest.approx(100.0 * tg.f[s] / g0.n)
        assert r["start_us"] == pytest.approx(s * 1.0)
    assert rows[0]["pct_activated"] == 100.0 and rows[-1]["mean_error"] == 0.0
    path = str(tmp_path / "conv.csv")
    diagnostics.write_csv(rows, path)
    with open(path) as fh:
        back = list(csv.DictReader(fh))
    assert tuple(back[0].keys()) == diagnostics.COLUMNS and len(back) == len(rows)
    assert float(back[-1]["mean_error"]) == 0.0
