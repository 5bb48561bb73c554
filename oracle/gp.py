"""FP64 oracle of the Bayesian optimal sampling proposal (test infrastructure).

Section 3.1 of arxiv 2309.03308: a Gaussian process with Matern covariance
models the correlation between the two bricks of a brick pair as a function of
a 6D position theta (3D in each brick); the Upper Confidence Bound mu +
kappa * sigma (kappa = 0.5, Section 6) is maximised to propose new samples;
continuous theta maps to voxels by probabilistic reparameterization,
P_i = floor(theta_i) + Bernoulli(theta_i - floor(theta_i)).

READINGS (the paper names the ingredients, not these settings):
  * Candidates: a fixed seeded pool of Q continuous positions per brick pair,
    uniform in [0, extent_d - 1] per axis; the first `per_round` pool
    entries are the initial random sample set.
  * Kernel: Matern nu = 5/2 with ARD length scales 0.25 * extent_d (voxels),
    signal variance = variance of the initial samples (floor 1e-6), noise
    variance 1e-4 * signal variance, constant prior mean = mean of the initial
    samples (or a supplied prior mean per pool entry).
  * Batch: per round, the top-M pool entries by UCB form a shortlist; `per_round`
    entries are picked greedily from it, each pick followed by the kriging
    believer update (the posterior covariance after observing the pick at its
    posterior mean: cov -= cov[:, c] cov[c, :] / (cov[c, c] + noise)).
  * Local picks (a project reading, `local_picks` > 0): from the second round
    on, the first `local_picks` proposals of a round are not taken from the
    pool but perturb the two best observations so far (by objective value,
    the earlier one on ties; proposal j uses incumbent j mod 2): theta =
    clip(theta_inc + local_scale * extent * z, 0, extent - 1) per axis, z
    standard normal (Box-Muller). They are evaluated, rounded and reduced like
    every proposal and can become incumbents, but the GP is conditioned on the
    pool proposals only.
  * Random numbers come from Philox4x64-10 through the oracle's own C
    implementation (`Oracle.philox`), with the counter layout documented in
    `pool_positions`, `bernoulli_voxels` and `local_theta`.
This module is plain numpy in FP64; scipy's cho_factor/cho_solve serve as the
Cholesky steps. Only tests and the benchmark's CPU leg may import it.
"""
from __future__ import annotations

import math

import numpy as np

SQRT5 = math.sqrt(5.0)
POOL_KEY = 0xB05B05
ROUND_KEY = 0xB0517D


def u24(words: np.ndarray) -> np.ndarray:
    """Uniform [0, 1) with 24 random bits (exact in fp32): top 24 bits of a word."""
    return ((words >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def pool_positions(orc, seed: int, rp: int, Q: int, ext_a, ext_b) -> np.ndarray:
    """Pool of Q positions [Q][6] (fp32) of region pair rp.

    Candidate c uses Philox blocks ctr = {c, rp, 0, 0} (axes 0-3) and
    {c, rp, 1, 0} (axes 4-5, first two words), key = {seed, POOL_KEY};
    theta_d = u24(word) * (extent_d - 1) in fp32.
    """
    ext = np.array(list(ext_a) + list(ext_b), dtype=np.float32)
    out = np.empty((Q, 6), np.float32)
    for c in range(Q):
        w = np.concatenate([orc.philox([c, rp, 0, 0], [seed, POOL_KEY]),
                            orc.philox([c, rp, 1, 0], [seed, POOL_KEY])[:2]])
        out[c] = u24(w) * (ext - np.float32(1))
    return out


def bernoulli_voxels(orc, seed: int, rp: int, rnd: int, j: int, theta: np.ndarray) -> np.ndarray:
    """Probabilistic reparameterization of one proposal (Section 3.1).

    Pick j of round rnd: u from blocks ctr = {j, rp, 2 + rnd, 0} and
    {j, rp, 2 + rnd, 1}, key = {seed, ROUND_KEY}; voxel_d = floor(theta_d) +
    (u_d < theta_d - floor(theta_d)), all fp32.
    """
    w = np.concatenate([orc.philox([j, rp, 2 + rnd, 0], [seed, ROUND_KEY]),
                        orc.philox([j, rp, 2 + rnd, 1], [seed, ROUND_KEY])[:2]])
    u = u24(w)
    th = theta.astype(np.float32)
    f = np.floor(th)
    frac = (th - f).astype(np.float32)
    return (f.astype(np.int64) + (u < frac)).astype(np.int64)


def box_muller(words: np.ndarray) -> np.ndarray:
    """Six standard normals from eight 64-bit words (FP64): for i = 0, 1, 2,
    u1 = (top 24 bits of w[2i] + 1) / 2^24 in (0, 1], u2 = top 24 bits of
    w[2i+1] / 2^24, z[2i] = sqrt(-2 ln u1) cos(2 pi u2), z[2i+1] = ... sin."""
    w = np.asarray(words, np.uint64)
    top = (w >> np.uint64(40)).astype(np.float64)
    z = np.empty(6)
    for i in range(3):
        u1 = (top[2 * i] + 1.0) * 2.0 ** -24
        u2 = top[2 * i + 1] * 2.0 ** -24
        rad = math.sqrt(-2.0 * math.log(u1))
        z[2 * i] = rad * math.cos(2.0 * math.pi * u2)
        z[2 * i + 1] = rad * math.sin(2.0 * math.pi * u2)
    return z


def local_theta(orc, seed: int, rp: int, rnd: int, j: int, theta_inc, ext, scale) -> np.ndarray:
    """Local proposal j of round rnd (a project reading): Philox blocks
    ctr = {j, rp, 2 + rnd, 2} and {j, rp, 2 + rnd, 3}, key = {seed, ROUND_KEY}
    give six normals z (`box_muller`); theta_d = clip(theta_inc_d + scale *
    ext_d * z_d, 0, ext_d - 1), in FP64."""
    w = np.concatenate([orc.philox([j, rp, 2 + rnd, 2], [seed, ROUND_KEY]),
                        orc.philox([j, rp, 2 + rnd, 3], [seed, ROUND_KEY])])
    z = box_muller(w)
    ext = np.asarray(ext, np.float64)
    return np.clip(np.asarray(theta_inc, np.float64) + scale * ext * z, 0.0, ext - 1.0)


def incumbents(thetas, values, count=2):
    """Indices of the `count` largest values (the earlier sample on ties)."""
    order = sorted(range(len(values)), key=lambda i: (-values[i], i))
    return order[:count]


def self_pair_fix(v, ext):
    """READING: in a self brick pair a sample never pairs a point with itself;
    when both voxels coincide, the second moves to the next point of the brick
    in enumeration order (x fastest), wrapping around."""
    v = np.array(v, np.int64)
    if tuple(v[:3]) == tuple(v[3:]):
        ex, ey, ez = ext
        l = (v[3] + ex * (v[4] + ey * v[5]) + 1) % (ex * ey * ez)
        v[3], v[4], v[5] = l % ex, (l // ex) % ey, l // (ex * ey)
    return v


def matern52(X1, X2, ell, sf2):
    """Matern nu = 5/2 covariance with ARD length scales (FP64)."""
    X1 = np.asarray(X1, np.float64) / ell
    X2 = np.asarray(X2, np.float64) / ell
    d2 = np.sum(X1 ** 2, 1)[:, None] + np.sum(X2 ** 2, 1)[None, :] - 2.0 * X1 @ X2.T
    r = np.sqrt(np.maximum(d2, 0.0))
    return sf2 * (1.0 + SQRT5 * r + 5.0 / 3.0 * r * r) * np.exp(-SQRT5 * r)


class GP:
    """Exact GP posterior (FP64) with a constant or per-pool prior mean."""

    def __init__(self, ell, sf2, sn2):
        self.ell, self.sf2, self.sn2 = np.asarray(ell, np.float64), float(sf2), float(sn2)

    def posterior(self, X, y, m_X, C, m_C):
        """Posterior mean and variance at C given observations y at X."""
        from scipy.linalg import cho_factor, cho_solve
        X = np.asarray(X, np.float64)
        if len(X) == 0:
            return np.asarray(m_C, np.float64).copy(), np.full(len(C), self.sf2)
        K = matern52(X, X, self.ell, self.sf2) + self.sn2 * np.eye(len(X))
        cf = cho_factor(K, lower=True)
        Ks = matern52(X, C, self.ell, self.sf2)
        alpha = cho_solve(cf, np.asarray(y, np.float64) - m_X)
        mu = m_C + Ks.T @ alpha
        var = self.sf2 - np.sum(Ks * cho_solve(cf, Ks), axis=0)
        return mu, var

    def posterior_cov(self, X, C):
        """Posterior covariance among the candidates C (no noise on C)."""
        from scipy.linalg import cho_factor, cho_solve
        Kcc = matern52(C, C, self.ell, self.sf2)
        if len(X) == 0:
            return Kcc
        K = matern52(X, X, self.ell, self.sf2) + self.sn2 * np.eye(len(X))
        cf = cho_factor(K, lower=True)
        Ks = matern52(X, C, self.ell, self.sf2)
        return Kcc - Ks.T @ cho_solve(cf, Ks)


def believer_picks(mu, cov, kappa, picks, sn2):
    """Greedy UCB picks with the kriging-believer covariance update.

    Returns the picked positions (indices into mu/cov) and the variances seen.
    Ties resolve to the smallest index.
    """
    cov = np.array(cov, np.float64, copy=True)
    taken = np.zeros(len(mu), bool)
    out = []
    for _ in range(picks):
        ucb = np.asarray(mu) + kappa * np.sqrt(np.maximum(np.diag(cov), 0.0))
        ucb[taken] = -np.inf
        c = int(np.argmax(ucb))
        out.append(c)
        taken[c] = True
        col = cov[:, c].copy()
        cov -= np.outer(col, col) / (col[c] + sn2)
    return out


def shortlist(ucb, selected, M):
    """Top-M unselected pool entries by UCB (ties: smaller index first)."""
    ucb = np.where(selected, -np.inf, ucb)
    order = np.lexsort((np.arange(len(ucb)), -ucb))
    return order[:M]


def bos_run(orc, objective, seed, rp, ext_a, ext_b, Q, per_round, rounds, kappa=0.5, M=128,
            prior=None, local_picks=0, local_scale=0.0625):
    """Plain BOS loop (FP64 GP refit from scratch every round) on one brick pair.

    objective(voxels [k][6] int) -> values [k]. Returns the pool, the pool
    indices observed per round (the GP's observations), the observed values,
    the voxel pairs, and every evaluated sample's theta and value in order.
    """
    pool = pool_positions(orc, seed, rp, Q, ext_a, ext_b)
    ext = np.array(list(ext_a) + list(ext_b), np.float64)
    ell = 0.25 * ext
    obs, ys, vox, rounds_picks = [], [], [], []
    th_all, y_all = [], []
    picks = list(range(per_round))
    gp = None
    m_pool = None
    for rnd in range(rounds):
        loc = []
        if rnd > 0:
            X = pool[obs]
            mu, var = gp.posterior(X, np.array(ys), m_pool[obs], pool, m_pool)
            selected = np.zeros(Q, bool)
            selected[obs] = True
            sl = shortlist(mu + kappa * np.sqrt(np.maximum(var, 0.0)), selected, M)
            cov = gp.posterior_cov(X, pool[sl])
            n_gp = per_round - local_picks
            picks = [int(sl[i]) for i in believer_picks(mu[sl], cov, kappa, n_gp, gp.sn2)]
            inc = incumbents(th_all, y_all)
            loc = [local_theta(orc, seed, rp, rnd, j, th_all[inc[j % len(inc)]], ext, local_scale)
                   for j in range(local_picks)]
        thetas = [np.asarray(t, np.float64) for t in loc] + [pool[c].astype(np.float64)
                                                               for c in picks]
        v = np.array([bernoulli_voxels(orc, seed, rp, rnd, j, np.float32(t))
                      for j, t in enumerate(thetas)])
        y = np.asarray(objective(v), np.float64)
        obs += picks
        ys += list(y[len(loc):])
        th_all += thetas
        y_all += list(y)
        vox.append(v)
        rounds_picks.append(picks)
        if rnd == 0:
            m = float(np.mean(y))
            sf2 = max(float(np.mean((y - m) ** 2)), 1e-6)
            gp = GP(ell, sf2, 1e-4 * sf2)
            m_pool = np.full(Q, m) if prior is None else np.asarray(prior, np.float64)
    return dict(pool=pool, picks=rounds_picks, y=np.array(ys), voxels=np.concatenate(vox),
                gp=gp, m_pool=m_pool, theta=np.array(th_all), y_all=np.array(y_all))
