"""A long batched BOS run against the FP64 GP oracle (Section 3.1): 20 rounds
of 32 proposals per region pair over a pool of 1024, so the GP holds up to
640 observations. This takes the tensor-core contractions of the GP through
many K blocks of observations, several pool tiles per region pair (both TMEM
accumulators reused), the full 128-entry shortlist, and the conditioning's
chunked gather of V[:, P] beyond its resident 512 rows; the posterior mean
and variance after the last round, and the last round's picks, are checked
against the oracle's."""
import numpy as np
import pytest

import gen
import oracle
from oracle import gp as ogp

pytestmark = pytest.mark.gpu

X, Y, Z, N = 40, 24, 6, 50
SEED, Q, R, T, M, KAPPA, K, BINS = 321, 1024, 32, 20, 128, 0.5, 5, 8


@pytest.fixture(scope="module")
def long_run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03308_gb300 import Context, build
    build.build()
    F = gen.field(33, X, Y, Z, N)
    ctx = Context(0)
    fid = ctx.load_field(F)
    rids = ctx.partition_regular(fid, 8, 8, 3)
    boxes = [ctx.region_info(r)[1] for r in rids]
    pairs = [(1, 9), (4, 4)]
    bos = ctx.bos_create(fid, [rids[a] for a, _ in pairs], [rids[b] for _, b in pairs], pool=Q,
                         per_round=R, rounds=T, shortlist=M, kappa=KAPPA, k=K, bins=BINS,
                         seed=SEED)
    bos.run(T)
    states = [bos.inspect(i) for i in range(len(pairs))]
    yield F, boxes, pairs, states
    bos.close()
    ctx.close()


def _replay(orc, F, boxes, pair, rp, st):
    ba, bb = boxes[pair[0]], boxes[pair[1]]
    ea = (ba[3] - ba[0], ba[4] - ba[1], ba[5] - ba[2])
    eb = (bb[3] - bb[0], bb[4] - bb[1], bb[5] - bb[2])
    pa, pb = [], []
    for i, c in enumerate(st["obs"]):
        rnd, j = divmod(i, R)
        v = ogp.bernoulli_voxels(orc, SEED, rp, rnd, j, st["pool"][c])
        if pair[0] == pair[1]:
            v = ogp.self_pair_fix(v, ea)
        pa.append((ba[0] + v[0]) + X * ((ba[1] + v[1]) + Y * (ba[2] + v[2])))
        pb.append((bb[0] + v[3]) + X * ((bb[1] + v[4]) + Y * (bb[2] + v[5])))
    y = orc.eval_pairs(F, oracle.MI_KSG, np.array(pa, np.uint32), np.array(pb, np.uint32), k=K,
                       bins=BINS)
    return ea, eb, y


def test_long_run_posterior_and_last_picks(long_run, orc):
    F, boxes, pairs, states = long_run
    for rp, (pair, st) in enumerate(zip(pairs, states)):
        assert len(st["obs"]) == R * T and len(set(st["obs"].tolist())) == R * T
        ea, eb, y = _replay(orc, F, boxes, pair, rp, st)
        assert np.abs(st["y"] - y).max() < 1e-5
        pool = st["pool"].astype(np.float64)
        m = float(np.mean(y[:R]))
        sf2 = max(float(np.mean((y[:R] - m) ** 2)), 1e-12)
        g = ogp.GP(0.25 * np.array(ea + eb, np.float64), sf2, 1e-4 * sf2)
        tol = 2e-3 * np.sqrt(sf2) + 1e-6
        # the last round's picks: in the shortlist and each a believer-UCB maximiser
        rnd = T - 1
        obs = st["obs"][:rnd * R]
        mu, var = g.posterior(pool[obs], y[:rnd * R], np.full(len(obs), m), pool, np.full(Q, m))
        ucb = mu + KAPPA * np.sqrt(np.maximum(var, 0))
        sel = np.zeros(Q, bool)
        sel[obs] = True
        sl = ogp.shortlist(ucb, sel, M)
        picks = list(st["obs"][rnd * R:])
        assert all(ucb[p] >= ucb[sl[-1]] - tol for p in picks)
        cand = np.array(list(sl) + [p for p in picks if p not in set(sl.tolist())])
        cov = g.posterior_cov(pool[obs], pool[cand])
        taken = np.zeros(len(cand), bool)
        for p in picks:
            i = int(np.nonzero(cand == p)[0][0])
            bu = mu[cand] + KAPPA * np.sqrt(np.maximum(np.diag(cov), 0))
            bu[taken] = -np.inf
            assert bu[i] >= bu.max() - tol, (p, bu[i], bu.max())
            taken[i] = True
            col = cov[:, i].copy()
            cov -= np.outer(col, col) / (col[i] + g.sn2)
        # the posterior after all 640 observations
        mu, var = g.posterior(pool[st["obs"]], y, np.full(R * T, m), pool, np.full(Q, m))
        assert np.abs(st["mu"] - mu).max() < 5e-3 * np.sqrt(sf2) + 1e-6
        assert np.abs(st["var"] - var).max() < 5e-3 * sf2 + 1e-9
