"""Schedule fuzzer for the asynchronous activation rules (CPU only).

The GPU sweep updates estimates in place while other vertices of the same
sweep read them, so a read may return the value a neighbour had when the sweep
began or the one it has written since.  This replays sweeps with random
evaluation orders and random stale reads and checks the claims the kernel
relies on (the in-place activation rules and why the asynchronous fixed point
is the coreness):

* the simple rule (push v iff new_u < x, Sec. III-B) always ends at the
  coreness;
* the refined rule of Sec. IV with the extra clause "or v is in the current
  frontier" always ends at the coreness;
* the refined rule alone (push v iff new_u < x <= old_u) does not: some
  schedule leaves an estimate above the coreness;
* the narrowed clause the kernel uses also always ends at the coreness: a
  vertex marks itself done once evaluated, and for a done vertex (or one not
  in the frontier) the refined test is applied to a value of est[v] read
  after seeing the mark (v's final value of the sweep);
* marks made later than the evaluation (the kernel's warp tier marks the
  vertices of one work grab together, after the grab) keep that rule safe;
* applying the refined test to the value read before the mark is unsafe;
* warm starts (dynamic maintenance): after deleting edges, starting from the
  old coreness with only the deleted edges' endpoints active, and after
  inserting b edges, starting from old core + b with every vertex active, both
  end at the new coreness.  A start above the degree is lowered to it, and
  that vertex and its neighbours start active.
"""
import random

import numpy as np
import pytest

import oracle
from tests import refimpl


def capped_hindex(vals, cap):
    return refimpl.hindex_sorted(vals, cap)


def run_async(n, adj, rule, rng, max_sweeps=10_000, start=None, active=None):
    est = [len(adj[v]) for v in range(n)] if start is None else \
        [min(int(start[v]), len(adj[v])) for v in range(n)]
    # a start above the degree is lowered to it: that vertex changed, so it
    # and its neighbours start active
    capped = set() if start is None else {v for v in range(n) if int(start[v]) > len(adj[v])}
    frontier = set(range(n)) if active is None else set(active)
    frontier |= capped | {w for v in capped for w in adj[v]}
    sweeps = 0
    while frontier:
        sweeps += 1
        assert sweeps < max_sweeps
        start = list(est)                     # values at the start of the sweep
        order = list(frontier)
        rng.shuffle(order)
        nxt = set()
        done = set()
        pending = []                          # deferred marks (refined_done_deferred)

        def read(v):                          # stale or fresh, at random
            return start[v] if rng.random() < 0.5 else est[v]

        for u in order:
            k = est[u]
            h = capped_hindex([read(v) for v in adj[u]], k)
            if rule == "refined_done_deferred":
                pending.append(u)             # marked with a later group, after its store
            else:
                done.add(u)
            if h >= k:
                continue
            est[u] = h
            for v in adj[u]:
                x = read(v)
                if rule == "simple":
                    push = h < x
                elif rule == "refined_frontier":
                    push = h < x and (x <= k or v in frontier)
                elif rule in ("refined_done", "refined_done_deferred"):
                    if h < x and x > k and v in frontier and v not in done:
                        push = True           # v may still be reading u's old value
                    elif h < x and x > k:
                        x2 = est[v]           # read again after seeing v done
                        push = h < x2 <= k
                    else:
                        push = h < x
                elif rule == "refined_done_stale":
                    push = h < x and (x <= k or (v in frontier and v not in done))
                else:                         # refined alone
                    push = h < x and x <= k
                if push:
                    nxt.add(v)
            if pending and (len(pending) >= 4 or rng.random() < 0.3):
                done.update(pending)
                pending = []
        frontier = nxt
    return est


def random_graph(rng, n, p):
    adj = [set() for _ in range(n)]
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < p:
                adj[a].add(b)
                adj[b].add(a)
    return [sorted(s) for s in adj]


def coreness(n, adj):
    src = [a for a in range(n) for b in adj[a]]
    dst = [b for a in range(n) for b in adj[a]]
    rp, col = oracle.csr_build(n, np.array(src, np.int32), np.array(dst, np.int32))
    return oracle.coreness(n, rp, col).tolist()


def test_safe_rules_always_reach_the_coreness():
    rng = random.Random(2024)
    for trial in range(250):
        n = rng.randint(2, 24)
        adj = random_graph(rng, n, rng.uniform(0.1, 0.6))
        core = coreness(n, adj)
        for rule in ("simple", "refined_frontier", "refined_done", "refined_done_deferred"):
            for _ in range(3):
                assert run_async(n, adj, rule, rng) == core, (trial, rule)


@pytest.mark.parametrize("rule", ["refined_alone", "refined_done_stale"])
def test_unsafe_refined_variants_can_fail_in_place(rule):
    rng = random.Random(7)
    failures = 0
    for trial in range(400):
        n = rng.randint(4, 20)
        adj = random_graph(rng, n, rng.uniform(0.2, 0.6))
        core = coreness(n, adj)
        for _ in range(4):
            est = run_async(n, adj, rule, rng)
            assert all(e >= c for e, c in zip(est, core))   # never below the coreness
            failures += est != core
    assert failures > 0


def test_warm_starts_after_deletions_and_insertions():
    rng = random.Random(31)
    for trial in range(200):
        n = rng.randint(3, 24)
        adj = random_graph(rng, n, rng.uniform(0.15, 0.6))
        core = coreness(n, adj)
        edges = [(a, b) for a in range(n) for b in adj[a] if a < b]
        # deletions: old coreness, endpoints active
        gone = rng.sample(edges, min(len(edges), rng.randint(1, 4)))
        adj2 = [set(x) for x in adj]
        for a, b in gone:
            adj2[a].discard(b)
            adj2[b].discard(a)
        adj2 = [sorted(x) for x in adj2]
        ends = {a for a, _ in gone} | {b for _, b in gone}
        for rule in ("simple", "refined_done"):
            assert run_async(n, adj2, rule, rng, start=core, active=ends) == coreness(n, adj2), trial
        # insertions: old coreness + b, everything active
        missing = [(a, b) for a in range(n) for b in range(a + 1, n) if b not in adj[a]]
        if not missing:
            continue
        new = rng.sample(missing, min(len(missing), rng.randint(1, 4)))
        adj3 = [set(x) for x in adj]
        for a, b in new:
            adj3[a].add(b)
            adj3[b].add(a)
        adj3 = [sorted(x) for x in adj3]
        start = [c + len(new) for c in core]
        for rule in ("simple", "refined_done"):
            assert run_async(n, adj3, rule, rng, start=start) == coreness(n, adj3), trial
