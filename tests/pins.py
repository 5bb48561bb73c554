"""Pins of the FP64 oracle against facts fixed outside it.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees with a closed form, a library routine, an invariant, a
hand-derived example or a statistical limit. ``test_oracle_pins.py`` runs them
on the oracle; ``test_oracle_plants.py`` runs them on builds of the oracle
with a planted mistake and requires them to fail.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def vec_pairs(o, kind, X, Y, **kw):
    """Measure between rows X[t] and Y[t] ([R][n] arrays) through the batch API."""
    X = np.asarray(X, dtype=np.float32)
    Y = np.asarray(Y, dtype=np.float32)
    R, n = X.shape
    F = np.empty((n, 2 * R), dtype=np.float32)
    F[:, 0::2] = X.T
    F[:, 1::2] = Y.T
    pa = np.arange(0, 2 * R, 2, dtype=np.uint32)
    return o.eval_pairs(F, kind, pa, pa + 1, **kw)


# ----------------------------------------------------------------------------- Pearson
def pin_pearson_affine(o):
    """r(x, a x + b) = sign(a) (PPMCC definition, Section 3.2)."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal((8, 50)).astype(np.float32)
    for a, b, s in ((2.0, 3.0, 1.0), (-0.5, 1.0, -1.0), (1.0, 0.0, 1.0)):
        y = (a * x.astype(np.float64) + b).astype(np.float32)
        r = vec_pairs(o, oracle.PEARSON, x, y)
        assert np.all(np.abs(r - s) < 1e-6), (a, b, r)


def pin_pearson_numpy(o):
    """Agreement with numpy.corrcoef, and symmetry."""
    rng = np.random.default_rng(12)
    x = rng.standard_normal((20, 37)).astype(np.float32)
    y = (0.4 * x + rng.standard_normal((20, 37)) + 5.0).astype(np.float32)
    r = vec_pairs(o, oracle.PEARSON, x, y)
    ref = np.array([np.corrcoef(x[i].astype(np.float64), y[i].astype(np.float64))[0, 1]
                    for i in range(20)])
    assert np.max(np.abs(r - ref)) < 1e-12, np.max(np.abs(r - ref))
    r2 = vec_pairs(o, oracle.PEARSON, y, x)
    assert np.array_equal(r, r2)


def pin_pearson_gaussian(o):
    """Bivariate normal: E[r] = rho - rho (1 - rho^2) / (2n) + O(1/n^2)."""
    n, R = 32, 4000
    for rho in (0.3, 0.8):
        a, b = gen.gaussian_pair(21, rho, n, R)
        r = vec_pairs(o, oracle.PEARSON, a, b)
        expect = rho - rho * (1 - rho * rho) / (2 * n)
        se = r.std() / math.sqrt(R)
        assert abs(r.mean() - expect) < 4 * se + 1e-3, (rho, r.mean(), expect, se)


def pin_pearson_constant(o):
    """READING: a zero-variance member vector has correlation 0."""
    x = np.ones((1, 16), np.float32)
    y = np.arange(16, dtype=np.float32)[None]
    assert vec_pairs(o, oracle.PEARSON, x, y)[0] == 0.0


# ----------------------------------------------------------------------------- Spearman
def pin_spearman_noties(o):
    """No ties: r_s = 1 - 6 sum d^2 / (n (n^2 - 1)) with integer rank differences."""
    rng = np.random.default_rng(13)
    n = 41
    for _ in range(10):
        x = rng.permutation(n).astype(np.float32) * 0.5 - 3.0
        y = rng.permutation(n).astype(np.float32) + 0.25
        rx = np.argsort(np.argsort(x))
        ry = np.argsort(np.argsort(y))
        d2 = int(np.sum((rx - ry) ** 2))
        expect = 1.0 - 6.0 * d2 / (n * (n * n - 1))
        r = vec_pairs(o, oracle.SPEARMAN, x[None], y[None])[0]
        assert abs(r - expect) < 1e-12, (r, expect)


def pin_spearman_scipy(o):
    """Ties averaged: agreement with scipy.stats.spearmanr."""
    from scipy.stats import spearmanr
    rng = np.random.default_rng(14)
    x = rng.integers(0, 6, (25, 30)).astype(np.float32)
    y = (x + rng.integers(0, 4, (25, 30))).astype(np.float32)
    r = vec_pairs(o, oracle.SPEARMAN, x, y)
    ref = np.array([spearmanr(x[i], y[i]).statistic for i in range(25)])
    assert np.max(np.abs(r - ref)) < 1e-12, np.max(np.abs(r - ref))


def pin_spearman_monotone(o):
    """Ranks are invariant under strictly increasing maps (bit-exact)."""
    rng = np.random.default_rng(15)
    v = rng.integers(-20, 20, (6, 33)).astype(np.float32)
    F1 = np.ascontiguousarray(v.T)
    F2 = np.ascontiguousarray((v.astype(np.float64) ** 3 + 7).astype(np.float32).T)
    pts = np.arange(6, dtype=np.uint32)
    assert np.array_equal(o.rank2(F1, pts), o.rank2(F2, pts))


def pin_spearman_gaussian(o):
    """Bivariate normal: E[r_s] = 6/(pi (n+1)) [asin(rho) + (n-2) asin(rho/2)] (Moran 1948)."""
    n, R = 32, 4000
    for rho in (0.4, 0.85):
        a, b = gen.gaussian_pair(22, rho, n, R)
        r = vec_pairs(o, oracle.SPEARMAN, a, b)
        expect = 6.0 / (math.pi * (n + 1)) * (math.asin(rho) + (n - 2) * math.asin(rho / 2))
        se = r.std() / math.sqrt(R)
        assert abs(r.mean() - expect) < 4 * se, (rho, r.mean(), expect, se)


# ----------------------------------------------------------------------------- binning / hist MI
def pin_bins_edges(o):
    """Equal-width bins over [min, max]: left edges b/B map to b, the maximum to B-1."""
    for B in (8, 16):
        edges = np.arange(B, dtype=np.float32) / B
        mids = (np.arange(B, dtype=np.float32) + 0.5) / B
        v = np.concatenate([edges, mids, [1.0]]).astype(np.float32)
        got = o.bins(v[:, None], np.array([0], np.uint32), B)[0]
        expect = np.concatenate([np.arange(B), np.arange(B), [B - 1]])
        assert np.array_equal(got, expect), (B, got)
        shifted = (v * 4 - 3).astype(np.float32)
        got2 = o.bins(shifted[:, None], np.array([0], np.uint32), B)[0]
        assert np.array_equal(got2, expect), (B, got2)
    c = np.full((12, 1), 2.5, np.float32)
    assert np.all(o.bins(c, np.array([0], np.uint32), 8) == 0)


def pin_hist_mi_sklearn(o):
    """MI of bin labels equals sklearn.metrics.mutual_info_score (nats)."""
    from sklearn.metrics import mutual_info_score
    rng = np.random.default_rng(16)
    for B in (8, 16):
        for _ in range(10):
            bx = rng.integers(0, B, 100).astype(np.uint8)
            by = ((bx.astype(int) + rng.integers(0, 3, 100)) % B).astype(np.uint8)
            mi = o.hist_mi_bins(bx, by, B)
            ref = mutual_info_score(bx, by)
            assert abs(mi - ref) < 1e-12, (mi, ref)


def pin_hist_mi_self(o):
    """MI(x, x) equals the entropy of the binned x."""
    from scipy.stats import entropy
    rng = np.random.default_rng(17)
    x = rng.standard_normal((5, 64)).astype(np.float32)
    mi = vec_pairs(o, oracle.MI_BINNED, x, x, bins=8)
    b = o.bins(np.ascontiguousarray(x.T), np.arange(5, dtype=np.uint32), 8)
    for i in range(5):
        h = entropy(np.bincount(b[i], minlength=8))
        assert abs(mi[i] - h) < 1e-12, (mi[i], h)


# ----------------------------------------------------------------------------- KSG
def pin_ksg_tiny(o):
    """Hand-derived n = 5 example (tests/golden/ksg_tiny_n5.json)."""
    g = json.load(open(os.path.join(GOLDEN, "ksg_tiny_n5.json")))
    for case in g["cases"]:
        mi, nx, ny, eps = o.ksg_vec(np.array(g["x"]), np.array(g["y"]), case["k"])
        assert list(eps) == case["eps"], (case["k"], eps)
        assert list(nx) == case["nx"], (case["k"], nx)
        assert list(ny) == case["ny"], (case["k"], ny)
        assert abs(mi - case["mi_num"] / case["mi_den"]) < 1e-12, (mi, case)


def pin_ksg_sklearn(o):
    """Agreement with sklearn's KSG (_compute_mi_cc) where fp32 differences are exact.

    Values are distinct multiples of 1/64 with |v| < 2^10, so every fp32
    difference is exact and sklearn's FP64 distances coincide with the fp32 ones.
    """
    from sklearn.feature_selection._mutual_info import _compute_mi_cc
    rng = np.random.default_rng(18)
    for n, k in ((50, 3), (100, 10), (200, 5)):
        for _ in range(3):
            x = (rng.permutation(4 * n)[:n] / 64.0).astype(np.float32)
            y = (x * 2 + rng.permutation(4 * n)[:n] / 64.0).astype(np.float32)
            mi, _, _, _ = o.ksg_vec(x, y, k)
            ref = _compute_mi_cc(x.astype(np.float64), y.astype(np.float64), k)
            assert ref > 0
            assert abs(mi - ref) < 1e-10, (n, k, mi, ref)


def pin_ksg_invariances(o):
    """Symmetry MI(X,Y) = MI(Y,X) bit-exact; member permutation permutes counts exactly."""
    rng = np.random.default_rng(19)
    x = rng.standard_normal(80).astype(np.float32)
    y = (x + rng.standard_normal(80)).astype(np.float32)
    m1, nx1, ny1, _ = o.ksg_vec(x, y, 4)
    m2, nx2, ny2, _ = o.ksg_vec(y, x, 4)
    assert m1 == m2 and np.array_equal(nx1, ny2) and np.array_equal(ny1, nx2)
    perm = rng.permutation(80)
    m3, nx3, ny3, _ = o.ksg_vec(x[perm], y[perm], 4)
    assert np.array_equal(nx3, nx1[perm]) and np.array_equal(ny3, ny1[perm])
    assert abs(m3 - m1) < 1e-12


def pin_ksg_gaussian(o):
    """Bivariate normal limit MI = -1/2 ln(1 - rho^2) (n = 1000, k = 10, 24 draws)."""
    n, R = 1000, 24
    for rho in (0.0, 0.3, 0.6, 0.9):
        a, b = gen.gaussian_pair(23, rho, n, R)
        mi = vec_pairs(o, oracle.MI_KSG, a, b, k=10)
        expect = -0.5 * math.log(1 - rho * rho)
        assert abs(mi.mean() - expect) < 0.03, (rho, mi.mean(), expect)


def pin_digamma(o):
    """psi at integers: scipy.special.digamma, psi(1) = -gamma, psi(m+1) = psi(m) + 1/m."""
    from scipy.special import digamma
    assert o.digamma_int(1) == -0.5772156649015329
    for m in (2, 3, 10, 100, 1000, 4096):
        assert abs(o.digamma_int(m) - digamma(m)) < 1e-13 * max(1.0, abs(digamma(m)))
    assert o.k_rule(100) == 3 and o.k_rule(1000) == 30 and o.k_rule(32) == 1


# ----------------------------------------------------------------------------- sampling
def pin_philox_numpy(o):
    """Philox4x64-10 equals numpy.random.Philox (which pre-increments its counter)."""
    rng = np.random.default_rng(20)
    for _ in range(20):
        ctr = rng.integers(1, 2**63, 4, dtype=np.uint64)
        key = rng.integers(0, 2**63, 2, dtype=np.uint64)
        before = ctr.copy()
        before[0] -= np.uint64(1)
        ref = np.random.Philox(counter=before, key=key).random_raw(4)
        assert np.array_equal(o.philox(ctr, key), ref)


def pin_sampler(o):
    """Sampled pairs stay in range, self pairs are ordered a < b, marginals are uniform."""
    ia, ib = o.sample_pairs(7, 0, 0, 37, 53, False, 200000)
    assert ia.max() < 37 and ib.max() < 53
    for c, m in ((np.bincount(ia, minlength=37), 37), (np.bincount(ib, minlength=53), 53)):
        e = 200000 / m
        chi2 = float(np.sum((c - e) ** 2 / e))
        assert chi2 < m + 6 * math.sqrt(2 * m), chi2
    sa, sb = o.sample_pairs(7, 1, 0, 20, 20, True, 50000)
    assert np.all(sa < sb) and sb.max() < 20
    ia2, ib2 = o.sample_pairs(7, 0, 100, 37, 53, False, 10)
    assert np.array_equal(ia2, ia[100:110]) and np.array_equal(ib2, ib[100:110])


# ----------------------------------------------------------------------------- region max
def pin_region_clusters(o):
    """Cluster fixture: the centres carry identical vectors, so the max Pearson is 1."""
    X, Y, Z, n = 12, 8, 2, 24
    F = gen.clusters(5, X, Y, Z, n, [(2, 2, 0, 3), (9, 5, 1, 3)])
    A = oracle.box_points(X, Y, Z, (0, 0, 0, 6, 8, 2))
    B = oracle.box_points(X, Y, Z, (6, 0, 0, 12, 8, 2))
    r = o.region_extremes(F, A, B, False, oracle.PEARSON)
    a, b = divmod(r["argmax"], len(B))
    assert abs(r["max"] - 1.0) < 1e-12 and (A[a], B[b]) == (2 + X * 2, 9 + X * (5 + Y)), r
    assert r["count"] == len(A) * len(B)
    s = o.region_extremes(F, A, A, True, oracle.PEARSON, want_values=True)
    assert s["count"] == len(A) * (len(A) - 1) // 2
    vals = s["values"].reshape(len(A), len(A))
    iu = np.triu_indices(len(A), 1)
    assert s["max"] == np.max(vals[iu]) and s["min"] == np.min(vals[iu])


# ----------------------------------------------------------------------------- python oracles
# The GP and MLP oracles are numpy modules; their pins take the oracle function
# itself so that test_oracle_plants.py can hand them a planted variant.
def pyo_self_pair_fix(fix):
    """Section 3.1 reparameterization in a self brick pair (reading: the second
    voxel of a coinciding sample moves to the next point of the brick in
    enumeration order, x fastest, wrapping)."""
    ext = (4, 3, 2)
    # hand-derived successors: (1,2,0) is point 9 -> point 10 = (2,2,0);
    # (3,0,0) is point 3 -> point 4 = (0,1,0) (x wraps into the next row);
    # (3,2,1) is the last point 23 -> point 0 (wraps to the first)
    for v, want in (((1, 2, 0), (2, 2, 0)), ((3, 0, 0), (0, 1, 0)), ((3, 2, 1), (0, 0, 0)),
                    ((0, 0, 1), (1, 0, 1))):
        got = tuple(int(t) for t in fix(list(v) + list(v), ext))
        assert got == tuple(v) + want, (v, got)
    pts = [(x, y, z) for z in range(ext[2]) for y in range(ext[1]) for x in range(ext[0])]
    succ = []
    for a in pts:
        for b in pts:
            got = tuple(int(t) for t in fix(list(a) + list(b), ext))
            assert got[:3] == a, (a, b, got)  # the first voxel never moves
            if a != b:
                assert got[3:] == b, (a, b, got)  # distinct voxels pass unchanged
            else:
                assert got[3:] != a and all(0 <= got[3 + d] < ext[d] for d in range(3)), got
                succ.append(got[3:])
    # the successors of all points are all points again (one cycle through the brick)
    assert sorted(succ) == sorted(pts)


def pyo_mlp_offsets(offsets):
    """The pair head's relative position (position_j - position_i) / (X, Y, Z),
    with point ids x + X (y + Y z)."""
    X, Y, Z = 10, 5, 4
    last = 9 + X * (4 + Y * 3)
    pi = np.array([0, 73, last, 12, 0], np.int64)
    pj = np.array([73, 0, 0, 12, last], np.int64)
    want = np.array([[0.3, 0.4, 0.25], [-0.3, -0.4, -0.25], [-0.9, -0.8, -0.75],
                     [0.0, 0.0, 0.0], [0.9, 0.8, 0.75]])
    got = offsets(X, Y, Z, pi, pj)
    assert np.abs(got - want).max() < 1e-15, got
    rng = np.random.default_rng(3)
    a = rng.integers(0, X * Y * Z, 200)
    b = rng.integers(0, X * Y * Z, 200)
    assert np.array_equal(offsets(X, Y, Z, a, b), -offsets(X, Y, Z, b, a))  # antisymmetry
    # points enumerated from a box decompose to that box's coordinates
    box = (2, 1, 1, 6, 4, 3)
    P = oracle.box_points(X, Y, Z, box)
    off = offsets(X, Y, Z, np.zeros(len(P), np.int64), P) * np.array([X, Y, Z])
    zz, yy, xx = np.meshgrid(np.arange(1, 3), np.arange(1, 4), np.arange(2, 6), indexing="ij")
    assert np.abs(off - np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1)).max() < 1e-12


def pyo_box_muller(bm):
    """Box-Muller on 24-bit uniforms: hand values and the standard normal's moments."""
    def words(tops):
        return np.array([np.uint64(t) << np.uint64(40) for t in tops], np.uint64)
    # top24 = 2^23 - 1 -> u1 = 1/2; top24 = 0 -> u2 = 0; top24 = 2^22 -> u2 = 1/4
    z = bm(words([2 ** 23 - 1, 0, 2 ** 23 - 1, 2 ** 22, 2 ** 24 - 1, 2 ** 23, 0, 0]))
    r = math.sqrt(2.0 * math.log(2.0))
    want = [r, 0.0, r * math.cos(math.pi / 2), r * math.sin(math.pi / 2), -0.0, 0.0]
    # u1 = 1 (top24 = 2^24 - 1) gives radius 0; u2 = 1/2 for the last pair
    assert np.abs(z - np.array(want)).max() < 1e-12, z
    rng = np.random.default_rng(5)
    zs = np.concatenate([bm(rng.integers(0, 2 ** 63, 8, dtype=np.int64).astype(np.uint64) * 2)
                         for _ in range(5000)])
    assert abs(zs.mean()) < 0.03 and abs(zs.var() - 1.0) < 0.05, (zs.mean(), zs.var())


def pyo_incumbents(inc):
    """The two largest values, the earlier sample on ties."""
    assert inc(None, [0.1, 0.5, 0.3, 0.5, 0.2]) == [1, 3]
    assert inc(None, [0.7, 0.1, 0.9]) == [2, 0]
    assert inc(None, [0.4]) == [0]


def pyo_local_theta(lt, orc):
    """Local proposals: centred on the incumbent, spread scale * extent per axis,
    clipped to the box."""
    ext = np.array([32, 32, 20, 20, 26, 20], np.float64)
    inc = np.array([10.0, 0.5, 18.5, 19.0, 3.0, 7.0])
    th = np.array([lt(orc, 3, 1, 2, j, inc, ext, 0.0625) for j in range(4000)])
    assert np.all(th >= 0) and np.all(th <= ext - 1)
    free = (inc > 4 * 0.0625 * ext) & (inc < ext - 1 - 4 * 0.0625 * ext)  # rarely clipped
    assert np.abs(th[:, free].mean(0) - inc[free]).max() < 0.1
    sd = th[:, free].std(0) / (0.0625 * ext[free])
    assert np.abs(sd - 1.0).max() < 0.06, sd
    assert np.mean(th[:, 1] == 0.0) > 0.3  # clipped at the low edge
    assert np.array_equal(lt(orc, 3, 1, 2, 7, inc, ext, 0.0625), lt(orc, 3, 1, 2, 7, inc, ext, 0.0625))


def py_pins():
    """(pin, oracle function) pairs of the python oracles."""
    from oracle import gp, mlp
    return [(pyo_self_pair_fix, gp.self_pair_fix), (pyo_mlp_offsets, mlp.offsets),
            (pyo_box_muller, gp.box_muller), (pyo_incumbents, gp.incumbents)]


ALL = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
