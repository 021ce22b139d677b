"""Readers for the hand-typed fixtures under tests/golden/."""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def lattice_table(q: int):
    """(c[q,3] int64, w[q] Fraction list) from tests/golden/lattice_d3q{q}.txt."""
    rows = []
    with open(os.path.join(GOLDEN, "lattice_d3q%d.txt" % q)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            i, cx, cy, cz, w = line.split()
            rows.append((int(i), int(cx), int(cy), int(cz), Fraction(w)))
    rows.sort()
    assert [r[0] for r in rows] == list(range(q))
    c = np.array([[r[1], r[2], r[3]] for r in rows], dtype=np.int64)
    w = [r[4] for r in rows]
    return c, w
