"""Pins of the aggregate oracle (oracle/agg.py, Section 3.3 mean / max trees)."""
import numpy as np

import gen
from oracle import agg


def test_constant_and_affine_fields():
    F = np.full((3, 4, 6, 5), 2.5, np.float32)
    assert np.all(agg.aggregate(F, 2, 2, 2) == 2.5)
    z, y, x = np.meshgrid(np.arange(4), np.arange(6), np.arange(8), indexing="ij")
    R = (1.0 + 2 * x + 3 * y - z).astype(np.float32)[None]
    M = agg.aggregate(R, 2, 3, 2)
    # the mean of an affine function over a full block is its value at the block centre
    cx, cy, cz = np.arange(4) * 2 + 0.5, np.arange(2) * 3 + 1.0, np.arange(2) * 2 + 0.5
    ref = 1.0 + 2 * cx[None, None, :] + 3 * cy[None, :, None] - cz[:, None, None]
    assert np.allclose(M[0], ref, rtol=0, atol=1e-6)


def test_ragged_blocks_conserve_the_sum_and_max_is_exact():
    F = gen.field(5, 7, 5, 3, 4)
    M = agg.aggregate(F, 3, 2, 2)
    assert M.shape == (4, 2, 3, 3)
    # weighted by the block point counts the means sum to the field's total
    zs, ys, xs = np.array([2, 1]), np.array([2, 2, 1]), np.array([3, 3, 1])
    cnt = zs[:, None, None] * ys[None, :, None] * xs[None, None, :]
    tot = (M.astype(np.float64) * cnt[None]).sum(axis=(1, 2, 3))
    assert np.allclose(tot, F.astype(np.float64).sum(axis=(1, 2, 3)), rtol=1e-6)
    X = agg.aggregate(F, 3, 2, 2, mode="max")
    assert X[1, 1, 2, 0] == F[1, 2:3, 4:5, 0:3].max()
    assert np.all(X >= M)
