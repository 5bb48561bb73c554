"""Pins of the FP64 GP / BOS oracle (Section 3.1) against scikit-learn's GP,
the kriging-believer identity, the reparameterization's expectation and a
Synth2-style analytic-maximum objective (Section 5.1)."""
import math

import numpy as np
import pytest

from oracle import gp as ogp


def test_matern_matches_sklearn():
    from sklearn.gaussian_process.kernels import Matern
    rng = np.random.default_rng(1)
    X1, X2 = rng.uniform(0, 10, (40, 6)), rng.uniform(0, 10, (30, 6))
    ell = np.array([2.0, 3.0, 1.0, 2.5, 4.0, 0.5])
    ref = 1.7 * Matern(length_scale=ell, nu=2.5)(X1, X2)
    assert np.abs(ogp.matern52(X1, X2, ell, 1.7) - ref).max() < 1e-12


def test_posterior_matches_sklearn():
    from sklearn.gaussian_process import GaussianProcessRegressor
    from sklearn.gaussian_process.kernels import ConstantKernel, Matern
    rng = np.random.default_rng(2)
    ell = np.array([2.0, 2.0, 1.0, 2.0, 2.0, 1.0])
    X, C = rng.uniform(0, 7, (50, 6)), rng.uniform(0, 7, (60, 6))
    y = np.sin(X.sum(1)) * 0.3 + 0.1
    m, sf2, sn2 = 0.05, 0.4, 1e-3
    g = ogp.GP(ell, sf2, sn2)
    mu, var = g.posterior(X, y, np.full(50, m), C, np.full(60, m))
    k = ConstantKernel(sf2, "fixed") * Matern(length_scale=ell, length_scale_bounds="fixed", nu=2.5)
    reg = GaussianProcessRegressor(kernel=k, alpha=sn2, optimizer=None).fit(X, y - m)
    rm, rs = reg.predict(C, return_std=True)
    assert np.abs(mu - (rm + m)).max() < 1e-9
    assert np.abs(var - rs ** 2).max() < 1e-9


def test_believer_update_is_conditioning():
    """Greedy rank-1 updates equal the posterior covariance after observing the picks."""
    rng = np.random.default_rng(3)
    ell = np.full(6, 2.0)
    g = ogp.GP(ell, 0.5, 1e-3)
    X, C = rng.uniform(0, 6, (20, 6)), rng.uniform(0, 6, (40, 6))
    cov = g.posterior_cov(X, C)
    mu = rng.normal(size=40) * 0.1
    picks = ogp.believer_picks(mu, cov, 0.5, 6, g.sn2)
    c = cov.copy()
    for p in picks:
        col = c[:, p].copy()
        c -= np.outer(col, col) / (col[p] + g.sn2)
    direct = g.posterior_cov(np.vstack([X, C[picks]]), C)
    assert np.abs(c - direct).max() < 1e-9
    assert len(set(picks)) == 6


def test_bernoulli_rounding_expectation(orc):
    theta = np.array([0.25, 3.5, 1.9, 6.0, 0.0, 2.75], np.float32)
    v = np.array([ogp.bernoulli_voxels(orc, 5, 0, 0, j, theta) for j in range(4000)])
    assert np.all(v >= np.floor(theta)) and np.all(v <= np.ceil(theta))
    assert np.abs(v.mean(0) - theta).max() < 0.04
    assert np.all(v[:, 3] == 6) and np.all(v[:, 4] == 0)


def test_pool_positions_in_range(orc):
    p = ogp.pool_positions(orc, 3, 7, 500, (32, 32, 20), (20, 26, 20))
    assert p.dtype == np.float32 and p.shape == (500, 6)
    hi = np.array([31, 31, 19, 19, 25, 19], np.float32)
    assert np.all(p >= 0) and np.all(p <= hi)


def synth2(rng, ext):
    """6-variate normal density over the 6D voxel domain (Section 5.1, Synth2)."""
    mean = rng.uniform(0, 1, 6) * (np.array(ext) - 1)
    A = rng.normal(size=(6, 6))
    S = A @ A.T / 6 + np.diag((np.array(ext) / 3.0) ** 2)
    Si = np.linalg.inv(S)
    norm = 1.0 / math.sqrt((2 * math.pi) ** 6 * np.linalg.det(S))

    def f(v):
        d = np.asarray(v, np.float64) - mean
        return norm * np.exp(-0.5 * np.einsum("ij,jk,ik->i", d, Si, d))
    return f


def test_bos_finds_synth2_maximum(orc):
    """BOS approaches the analytic objective's maximum and beats random sampling.

    Normalised error (max - found) / (max - min) as in Section 5.3, 96 samples
    per brick pair, 6 brick pairs. Thresholds calibrated once on this oracle
    (observed median 0.14, max 0.18; random sampling with the same budget:
    mean 0.35) and frozen; the fixed candidate pool bounds how close the
    proposals can get.
    """
    ext_a, ext_b = (8, 8, 4), (8, 8, 4)
    ext = list(ext_a) + list(ext_b)
    grid = np.stack(np.meshgrid(*[np.arange(e) for e in ext], indexing="ij"), -1).reshape(-1, 6)
    errs, rand = [], []
    for t in range(6):
        f0 = synth2(np.random.default_rng(40 + t), ext)
        vals = f0(grid)
        hi = vals.max()
        lo = vals.min() / hi

        def f(v):
            return f0(v) / hi
        r = ogp.bos_run(orc, f, 11, t, ext_a, ext_b, Q=1024, per_round=16, rounds=6)
        rr = ogp.bos_run(orc, f, 11, t, ext_a, ext_b, Q=1024, per_round=96, rounds=1)
        errs.append((1.0 - r["y"].max()) / (1.0 - lo))
        rand.append((1.0 - rr["y"].max()) / (1.0 - lo))
    errs = np.array(errs)
    assert np.median(errs) < 0.2 and errs.max() < 0.3, errs
    assert errs.mean() < np.mean(rand), (errs, rand)


def test_bos_local_picks_on_synth2(orc):
    """With local picks (8 of 16 per round around the two incumbents) BOS reaches
    the analytic maximum of the Synth2-style objective at least as closely as
    without, on the same six brick pairs; local samples are evaluated but the
    GP is conditioned on the pool proposals only."""
    ext_a, ext_b = (8, 8, 4), (8, 8, 4)
    ext = list(ext_a) + list(ext_b)
    grid = np.stack(np.meshgrid(*[np.arange(e) for e in ext], indexing="ij"), -1).reshape(-1, 6)
    plain, local = [], []
    for t in range(6):
        f0 = synth2(np.random.default_rng(40 + t), ext)
        vals = f0(grid)
        hi = vals.max()
        lo = vals.min() / hi

        def f(v):
            return f0(v) / hi
        r0 = ogp.bos_run(orc, f, 11, t, ext_a, ext_b, Q=1024, per_round=16, rounds=6)
        r1 = ogp.bos_run(orc, f, 11, t, ext_a, ext_b, Q=1024, per_round=16, rounds=6,
                         local_picks=8, local_scale=0.0625)
        assert len(r1["y_all"]) == 16 * 6 and len(r1["y"]) == 16 + 5 * 8
        assert np.array_equal(r1["y_all"][:16], r1["y"][:16])  # round 0: pool samples only
        plain.append((1.0 - r0["y_all"].max()) / (1.0 - lo))
        local.append((1.0 - r1["y_all"].max()) / (1.0 - lo))
    assert np.mean(local) <= np.mean(plain) + 0.01, (local, plain)
