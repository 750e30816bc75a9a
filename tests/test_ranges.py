"""The batch engine's first-fit range allocator (csrc/ranges.h, host C++),
compiled with g++ and driven through seeded random take/give sequences against
a plain Python model: the same offsets, the same largest free range, the same
used count and peak, live ranges never overlapping, and a fully coalesced free
list once everything is given back (also after a reset)."""
import os
import random
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include "ranges.h"
#include <cstdio>
int main() {
    kc::Ranges r;
    char op;
    long long a, b;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'R' && std::scanf("%lld", &a) == 1) r.reset(a);
        else if (op == 'T' && std::scanf("%lld", &a) == 1) std::printf("%lld\n", r.take(a));
        else if (op == 'G' && std::scanf("%lld %lld", &a, &b) == 2) r.give(a, b);
        else if (op == 'S') std::printf("%lld %lld %lld\n", r.largest(), r.used(), r.peak());
    }
    return 0;
}
"""


class Model:
    def __init__(self):
        self.free, self.used, self.peak = [], 0, 0

    def reset(self, cap):
        self.free, self.used = ([(0, cap)] if cap > 0 else []), 0

    def take(self, n):
        if n <= 0:
            return 0
        for i, (at, ln) in enumerate(self.free):
            if ln >= n:
                self.free[i:i + 1] = [(at + n, ln - n)] if ln > n else []
                self.used += n
                self.peak = max(self.peak, self.used)
                return at
        return -1

    def give(self, at, n):
        if n <= 0:
            return
        self.used -= n
        self.free.append((at, n))
        self.free.sort()
        merged = []
        for s, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == s:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((s, ln))
        self.free = merged

    def stats(self):
        return (max((ln for _, ln in self.free), default=0), self.used, self.peak)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("ranges")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I",
                    os.path.join(ROOT, "paper_2512_00233_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True)
    return str(exe)


@pytest.mark.parametrize("seed", range(6))
def test_ranges_match_model(driver, seed):
    rng = random.Random(seed)
    cap = rng.choice([64, 1000, 1 << 20])
    m = Model()
    ops, expect, live = [f"R {cap}"], [], []
    m.reset(cap)
    for step in range(3000):
        if step == 1500:                      # everything back, then a reset mid-run
            for at, n in live:
                ops.append(f"G {at} {n}")
                m.give(at, n)
            live = []
            ops.append("S")
            expect.append(m.stats())
            assert m.stats()[0] == cap and m.stats()[1] == 0
            ops.append(f"R {cap}")
            m.reset(cap)
        if live and rng.random() < 0.45:
            at, n = live.pop(rng.randrange(len(live)))
            ops.append(f"G {at} {n}")
            m.give(at, n)
        else:
            n = rng.randint(0, max(1, cap // 12))
            ops.append(f"T {n}")
            at = m.take(n)
            expect.append(at)
            if at >= 0 and n > 0:
                assert all(at + n <= a or a + b <= at for a, b in live)   # no overlap
                assert 0 <= at and at + n <= cap
                live.append((at, n))
        if step % 97 == 0:
            ops.append("S")
            expect.append(m.stats())
    for at, n in live:
        ops.append(f"G {at} {n}")
        m.give(at, n)
    ops.append("S")
    expect.append(m.stats())
    assert m.stats()[:2] == (cap, 0)
    out = subprocess.run([driver], input="\n".join(ops) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    got = []
    for line in out:
        if not line.strip():
            continue
        parts = [int(x) for x in line.split()]
        got.append(parts[0] if len(parts) == 1 else tuple(parts))
    assert got == expect
