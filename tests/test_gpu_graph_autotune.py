"""CUDA-graph replay of a run (KCORE_GRAPH) and the launch-knob autotuner.

Both change only how the same kernels are issued or configured, so the
coreness must equal the oracle's exactly on every replay and for every tuned
configuration.
"""
import json

import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K
from paper_2512_00233_gb300 import autotune

pytestmark = pytest.mark.gpu


def oracle_core(g0):
    rp, col = oracle.csr_build(g0.n, g0.src, g0.dst)
    return rp, col, oracle.coreness(g0.n, rp, col)


def test_graph_replay_matches_oracle_and_counts_launches():
    import torch
    g0 = graphgen.rmat(1 << 14, 16 << 14, 0.57, 0.19, 0.19, seed=31)
    _, _, core = oracle_core(g0)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        out = torch.full((g0.n,), -1, dtype=torch.int32, device="cuda")
        g.run(out=out, graph=True)                           # capture + first replay
        np.testing.assert_array_equal(out.cpu().numpy(), core)
        st0 = g.stats()
        assert st0["status"] == 0 and st0["ms_sweep"] > 0 and st0["sweeps"] > 1
        for _ in range(3):
            out.fill_(-1)
            before = K.lib().kcore_kernel_launches()
            g.run(out=out, graph=True)
            after = K.lib().kcore_kernel_launches()
            np.testing.assert_array_equal(out.cpu().numpy(), core)
            assert after - before == 1                       # the persistent sweep launch
            st = g.stats()
            assert st["status"] == 0 and st["sweeps"] > 1 and st["ms_sweep"] > 0
        # a new output pointer, then mixing with direct runs
        out2 = torch.empty(g0.n, dtype=torch.int32, device="cuda")
        g.run(out=out2, graph=True)
        np.testing.assert_array_equal(out2.cpu().numpy(), core)
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
        out.fill_(-1)
        g.run(out=out, graph=True)
        np.testing.assert_array_equal(out.cpu().numpy(), core)


@pytest.mark.parametrize("refined", [False, True])
def test_graph_replay_sync_mode_and_options(refined):
    import torch
    g0 = graphgen.damaged_grid(256, seed=4)
    rp, col, core = oracle_core(g0)
    rounds, _, fr, _ = oracle.montresor_sync(g0.n, rp, col, refined=refined, record=100000)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        out = torch.empty(g0.n, dtype=torch.int32, device="cuda")
        for _ in range(2):
            g.run(out=out, graph=True, sync_mode=True, refined=refined)
            np.testing.assert_array_equal(out.cpu().numpy(), core)
            assert g.stats()["sweeps"] == rounds
            f, _, _ = g.trace()
            np.testing.assert_array_equal(f, fr)
        # options changed after capture: the graph is captured again
        g.set_options(K.default_options(t_lo=4, t_hi=32, block=256, tail_max=-1))
        out.fill_(-1)
        g.run(out=out, graph=True)
        np.testing.assert_array_equal(out.cpu().numpy(), core)
        g.set_options(K.default_options(max_sweeps=2))
        g.run(out=out, graph=True, check_status=False)
        assert g.last_status == K.KCORE_ERR_NOT_CONVERGED


def test_graph_replay_async_on_caller_stream():
    import torch
    g0 = graphgen.er(50_000, 400_000, seed=6)
    _, _, core = oracle_core(g0)
    s = torch.cuda.Stream()
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        out = torch.empty(g0.n, dtype=torch.int32, device="cuda")
        for _ in range(3):
            with torch.cuda.stream(s):
                out.fill_(-1)                            # ordered before the replay
                g.run(out=out, graph=True, wait=False, stream=s)
                res = out.clone()                        # ordered after it
            assert g.wait() == K.KCORE_OK
            s.synchronize()
            np.testing.assert_array_equal(res.cpu().numpy(), core)


def test_graph_flag_needs_device_output():
    g0 = graphgen.er(1000, 4000, seed=1)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        with pytest.raises(K.KCoreError) as e:
            g.run(device=False, graph=True)
        assert e.value.status == K.KCORE_ERR_INVALID


def test_autotune_keeps_results_and_caches(tmp_path):
    g0 = graphgen.damaged_grid(512, seed=8)
    _, _, core = oracle_core(g0)
    cache = str(tmp_path / "tune.json")
    space = {"t_lo": [8, 16], "block": [256, 512], "tail_max": [256, 1024]}
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        opts, trials = autotune.autotune(g, reps=2, passes=1, space=space, cache=cache)
        assert len(trials) >= 1 + 3
        assert all(ms > 0 for _, _, ms in trials)
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
        key = autotune.shape_key(g)
        with open(cache) as f:
            data = json.load(f)
        assert key in data and data[key]["ms_sweep"] > 0
        again = autotune.tuned_options(g, cache)
        for k in space:
            assert getattr(again, k) == getattr(opts, k)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst, options=again) as g:
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
