"""Writes tests/golden/two_triangles_4x4.json from the exact rational reference
(oracle/exact.py) only: the mixed coupling matrix B (Sec. 2.3, mortar integrals)
of two triangles on a 4x4 nodal Q1 grid over [0,1]^2, as exact fractions."""
import json
import os
import sys
from fractions import Fraction as Fr

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import exact  # noqa: E402


def build() -> dict:
    """The stored fixture's content, computed from oracle/exact.py."""
    import math
    coords = [[0.30, 0.20], [0.80, 0.35], [0.45, 0.70], [0.90, 0.85]]
    elems = [[0, 1, 2], [1, 3, 2]]
    n, h = 4, 0.25
    B = {}
    for e, tri in enumerate(elems):
        V = [coords[v] for v in tri]
        lo = [min(p[k] for p in V) for k in range(2)]
        hi = [max(p[k] for p in V) for k in range(2)]
        for j in range(math.floor(lo[1] / h), math.ceil(hi[1] / h)):
            for i in range(math.floor(lo[0] / h), math.ceil(hi[0] / h)):
                blk, vol = exact.pair_block_exact(2, V, [i * h, j * h], [h, h])
                if vol == 0:
                    continue
                for a in range(3):
                    for b in range(4):
                        col = (i + (b & 1)) + (n + 1) * (j + (b >> 1))
                        key = (tri[a], col)
                        B[key] = B.get(key, Fr(0)) + blk[a][b]
    return dict(coords=coords, elems=elems, ncell=[n, n], h=[h, h], origin=[0.0, 0.0],
                B=[[r, c, str(v)] for (r, c), v in sorted(B.items())],
                source="exact rational vertex enumeration + Grundmann-Moeller (oracle/exact.py)")


if __name__ == "__main__":
    out = build()
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "two_triangles_4x4.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(len(out["B"]), "entries")
