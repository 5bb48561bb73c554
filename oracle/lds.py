"""FP64/integer oracle of the quasi-random pair samplers (test infrastructure;
only tests, the smoke check and the benchmark's CPU leg may import it).

Section 3.1 names quasi-random low-discrepancy sequences -- Halton and
plastic-type sequences -- as alternatives to uniform random samples in the 6D
space of a brick pair. Definitions taken here (the paper gives no formulas):

  point index j = first + t + 1 for pair t (the all-zero point j = 0 skipped)
  Halton (Halton 1960): u_d = radical inverse of j in base (2, 3, 5, 7, 11, 13)[d],
      u_d = N_d / b^K with N_d the K base-b digits of j in reverse order; the
      voxel coordinate is c_d = floor(N_d * ext_d / b^K), exact integer arithmetic.
  R6 (Roberts' generalisation of the plastic-number sequence to 6 dimensions):
      phi = the real root of x^7 = x + 1, alpha_d = phi^-(d+1) rounded to the
      nearest double; u_d = frac(0.5 + j * alpha_d) evaluated in IEEE double
      (product, sum and floor each rounded once); c_d = min(floor(u_d * ext_d),
      ext_d - 1).
  Coordinates (c_0, c_1, c_2) index region A's box and (c_3, c_4, c_5) region
  B's; a, b are region-local indices x + ext_x (y + ext_y z). For a self
  region pair: if a == b then b = (b + 1) mod |A|; then ordered so a < b.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

HALTON_BASES = (2, 3, 5, 7, 11, 13)


def radical_inverse(j: int, b: int) -> Fraction:
    """Digits of j in base b mirrored behind the radix point (exact)."""
    num, den = 0, 1
    while j > 0:
        j, d = divmod(j, b)
        num = num * b + d
        den *= b
    return Fraction(num, den)


def halton_coord(j: int, b: int, ext: int) -> int:
    f = radical_inverse(j, b)
    return (f.numerator * ext) // f.denominator


def r6_alphas() -> list[float]:
    """alpha_d = phi^-(d+1), phi the real root of x^7 - x - 1, nearest doubles."""
    lo, hi = Fraction(1), Fraction(2)
    for _ in range(200):  # bisection to 2^-200
        mid = (lo + hi) / 2
        if mid ** 7 - mid - 1 > 0:
            hi = mid
        else:
            lo = mid
    phi = (lo + hi) / 2
    return [float(1 / phi ** (d + 1)) for d in range(6)]


def r6_coord(j: int, alpha: float, ext: int) -> int:
    u = 0.5 + float(j) * alpha  # IEEE double: product, then sum
    u = u - math.floor(u)
    return min(int(math.floor(u * float(ext))), ext - 1)


def sample_pairs_lds(kind: str, box_a, box_b, self_pair: bool, first: int, n: int):
    """Region-local (a, b) index arrays for pairs t = 0 .. n-1."""
    ext = [box_a[3] - box_a[0], box_a[4] - box_a[1], box_a[5] - box_a[2],
           box_b[3] - box_b[0], box_b[4] - box_b[1], box_b[5] - box_b[2]]
    na = ext[0] * ext[1] * ext[2]
    alphas = r6_alphas() if kind == "r6" else None
    a_out = np.empty(n, np.int64)
    b_out = np.empty(n, np.int64)
    for t in range(n):
        j = first + t + 1
        if kind == "halton":
            c = [halton_coord(j, HALTON_BASES[d], ext[d]) for d in range(6)]
        elif kind == "r6":
            c = [r6_coord(j, alphas[d], ext[d]) for d in range(6)]
        else:
            raise ValueError(kind)
        a = c[0] + ext[0] * (c[1] + ext[1] * c[2])
        b = c[3] + ext[3] * (c[4] + ext[4] * c[5])
        if self_pair:
            if a == b:
                b = (b + 1) % na
            a, b = min(a, b), max(a, b)
        a_out[t], b_out[t] = a, b
    return a_out, b_out
