"""Convergence diagnostics (Fig. 4 / Fig. 5 quantities) against the oracle.

In synchronous mode every round is deterministic, so the per-round mean error
and activation counts must equal the oracle's Jacobi iteration exactly; in
asynchronous mode the error must fall monotonically to zero.
"""
import csv

import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K
from paper_2512_00233_gb300 import diagnostics

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("refined", [False, True])
def test_sync_rounds_match_oracle(refined):
    g0 = graphgen.damaged_grid(96, seed=3)
    rp, col = oracle.csr_build(g0.n, g0.src, g0.dst)
    core = oracle.coreness(g0.n, rp, col)
    rounds, _, fr, _ = oracle.montresor_sync(g0.n, rp, col, refined=refined, record=100000)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        out = g.run(sync_mode=True, refined=refined, device=False)
        np.testing.assert_array_equal(out, core)
        rows = diagnostics.convergence(g, out)
    assert len(rows) == rounds
    for s, r in enumerate(rows):
        _, est_s, _, _ = oracle.montresor_sync(g0.n, rp, col, max_rounds=s + 1, refined=refined)
        expect = float((est_s.astype(np.int64) - core).sum()) / g0.n
        assert r["mean_error"] == pytest.approx(expect, abs=0.0), s
        assert r["activated"] == fr[s]
    assert rows[-1]["mean_error"] == 0.0


def test_async_error_falls_to_zero_and_csv(tmp_path):
    g0 = graphgen.rmat(1 << 14, 16 << 14, 0.57, 0.19, 0.19, seed=8)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        out = g.run(device=False)
        rows = diagnostics.convergence(g, out)
    err = [r["mean_error"] for r in rows]
    assert rows[0]["pct_activated"] == 100.0
    assert all(a >= b for a, b in zip(err, err[1:]))
    assert err[-1] == 0.0 and err[0] > 0.0
    path = str(tmp_path / "conv.csv")
    diagnostics.write_csv(rows, path)
    with open(path) as fh:
        got = list(csv.DictReader(fh))
    assert len(got) == len(rows) and tuple(got[0].keys()) == diagnostics.COLUMNS
