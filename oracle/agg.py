"""Oracle of the spatial aggregates (test infrastructure; only tests, the smoke
check and the benchmark's CPU leg may import it).

Section 3.3: a hierarchical representation stores, per brick and ensemble
member, the mean (mean-tree) or the maximum (max-tree) of the values at the
grid points the brick covers; sampling then runs on these aggregates. One
level is computed here: blocks of bx x by x bz grid points (the last block of
an axis is smaller when the extent is not a multiple), the mean as the
correctly rounded fp32 value of the exact sum divided by the block's point
count (math.fsum), the maximum exactly.
"""
from __future__ import annotations

import math

import numpy as np


def aggregate(F: np.ndarray, bx: int, by: int, bz: int, mode: str = "mean") -> np.ndarray:
    """F [n][Z][Y][X] fp32 -> [n][ceil(Z/bz)][ceil(Y/by)][ceil(X/bx)] fp32."""
    n, Z, Y, X = F.shape
    Zc, Yc, Xc = -(-Z // bz), -(-Y // by), -(-X // bx)
    out = np.empty((n, Zc, Yc, Xc), np.float32)
    for m in range(n):
        for k in range(Zc):
            for j in range(Yc):
                for i in range(Xc):
                    blk = F[m, k * bz:(k + 1) * bz, j * by:(j + 1) * by, i * bx:(i + 1) * bx]
                    if mode == "mean":
                        vals = [float(v) for v in blk.ravel()]
                        out[m, k, j, i] = np.float32(math.fsum(vals) / len(vals))
                    else:
                        out[m, k, j, i] = blk.max()
    return out
