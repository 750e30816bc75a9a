"""Reader for the hand-derived fixtures in tests/golden/."""
from __future__ import annotations

import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(path: str) -> dict:
    sect, out = None, {"edges": [], "name": os.path.basename(path)}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head = line.split()
            if head[0] == "n":
                out["n"] = int(head[1])
                continue
            if head[0] in ("edges", "coreness", "row_ptr", "col"):
                sect = head[0]
                continue
            vals = [int(x) for x in head]
            if sect == "edges":
                out["edges"].append((vals[0], vals[1]))
            else:
                out.setdefault(sect, []).extend(vals)
    e = np.array(out["edges"], dtype=np.int32).reshape(-1, 2)
    out["src"], out["dst"] = e[:, 0].copy(), e[:, 1].copy()
    return out


def all_fixtures() -> list[dict]:
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]
