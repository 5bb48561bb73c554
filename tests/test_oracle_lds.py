"""Pins of the quasi-random pair sampler oracle (oracle/lds.py) against the
definitions of the Halton and R-sequences (Section 3.1 names both families)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import lds


def test_radical_inverse_hand_values():
    assert lds.radical_inverse(1, 2) == Fraction(1, 2)
    assert lds.radical_inverse(2, 2) == Fraction(1, 4)
    assert lds.radical_inverse(3, 2) == Fraction(3, 4)
    assert lds.radical_inverse(6, 2) == Fraction(3, 8)   # 110 -> 0.011
    assert lds.radical_inverse(1, 3) == Fraction(1, 3)
    assert lds.radical_inverse(4, 3) == Fraction(4, 9)   # 11 -> 0.11
    assert lds.radical_inverse(5, 3) == Fraction(7, 9)   # 12 -> 0.21
    assert lds.radical_inverse(13, 13) == Fraction(1, 169)


@pytest.mark.parametrize("b,k", [(2, 10), (3, 6), (5, 4), (13, 2)])
def test_halton_stratifies_each_coordinate(b, k):
    """j = 0 .. b^k - 1 puts exactly one point in each interval of width b^-k
    (the van der Corput property)."""
    cells = sorted(lds.halton_coord(j, b, b ** k) for j in range(b ** k))
    assert cells == list(range(b ** k))


def test_r6_root_and_constants():
    roots = np.roots([1, 0, 0, 0, 0, 0, -1, -1])
    phi = max(r.real for r in roots if abs(r.imag) < 1e-12)
    al = lds.r6_alphas()
    assert abs(al[0] - 1 / phi) < 1e-14
    assert all(abs(al[d] - phi ** -(d + 1)) < 1e-14 for d in range(6))
    assert all(1 > al[d] > al[d + 1] > 0 for d in range(5))
    p = 1 / al[0]
    assert abs(p ** 7 - p - 1) < 1e-12


def test_r6_is_evenly_spread():
    """A Kronecker sequence with these constants fills each coordinate's 64
    cells far more evenly than random numbers over 2^16 points: every cell
    within 5 % of the mean and 1.5 % on average over the six coordinates
    (independent uniform numbers deviate by ~7 % in their worst cell)."""
    al = lds.r6_alphas()
    n = 1 << 16
    worst = []
    for d in range(6):
        c = np.array([lds.r6_coord(j, al[d], 64) for j in range(1, n + 1)])
        h = np.bincount(c, minlength=64)
        worst.append(np.abs(h - n / 64).max() / (n / 64))
    assert max(worst) < 0.05 and np.mean(worst) < 0.015, worst


@pytest.mark.parametrize("kind", ["halton", "r6"])
def test_pair_mapping_ranges_and_self_order(kind):
    box_a, box_b = (2, 3, 0, 9, 8, 3), (0, 0, 1, 4, 5, 4)
    a, b = lds.sample_pairs_lds(kind, box_a, box_b, False, 17, 500)
    assert a.min() >= 0 and a.max() < 7 * 5 * 3 and b.min() >= 0 and b.max() < 4 * 5 * 3
    a, b = lds.sample_pairs_lds(kind, box_a, box_a, True, 0, 500)
    assert np.all(a < b) and b.max() < 7 * 5 * 3
