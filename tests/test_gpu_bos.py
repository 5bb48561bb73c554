"""Batched Bayesian optimal sampling on the GPU against the FP64 GP oracle
(Section 3.1): pool positions bit-exact, rounded voxels and measured values,
every proposal a valid UCB / kriging-believer choice of the oracle's posterior,
the final posterior mean and variance, graph replay identical to direct
launches."""
import numpy as np
import pytest

import gen
import oracle
from oracle import gp as ogp

pytestmark = pytest.mark.gpu

X, Y, Z, N = 40, 24, 6, 50
SEED, Q, R, T, M, KAPPA, K, BINS = 123, 256, 8, 4, 32, 0.5, 5, 8


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03308_gb300 import Context, build
    build.build()
    F = gen.field(31, X, Y, Z, N)
    ctx = Context(0)
    fid = ctx.load_field(F)
    rids = ctx.partition_regular(fid, 8, 8, 3)
    boxes = [ctx.region_info(r)[1] for r in rids]
    pairs = [(0, 7), (3, 3), (5, 20)]
    rp_a = [rids[a] for a, _ in pairs]
    rp_b = [rids[b] for _, b in pairs]
    runs = {}
    for graph in (True, False):
        bos = ctx.bos_create(fid, rp_a, rp_b, pool=Q, per_round=R, rounds=T, shortlist=M,
                             kappa=KAPPA, k=K, bins=BINS, seed=SEED)
        bos.run(T, use_graph=graph)
        runs[graph] = (bos, [bos.inspect(i) for i in range(len(pairs))], bos.results())
    yield F, boxes, pairs, runs
    for bos, _, _ in runs.values():
        bos.close()
    ctx.close()


def ext_of(box):
    return (box[3] - box[0], box[4] - box[1], box[5] - box[2])


def point_ids(box_a, box_b, v):
    a = (box_a[0] + v[0]) + X * ((box_a[1] + v[1]) + Y * (box_a[2] + v[2]))
    b = (box_b[0] + v[3]) + X * ((box_b[1] + v[4]) + Y * (box_b[2] + v[5]))
    return a, b


def replay(orc, F, boxes, pair, rp, st):
    """Oracle evaluation of the GPU's observed samples, in order."""
    ba, bb = boxes[pair[0]], boxes[pair[1]]
    ea, eb = ext_of(ba), ext_of(bb)
    pa, pb = [], []
    for i, c in enumerate(st["obs"]):
        rnd, j = divmod(i, R)
        v = ogp.bernoulli_voxels(orc, SEED, rp, rnd, j, st["pool"][c])
        if pair[0] == pair[1]:
            v = ogp.self_pair_fix(v, ea)
        a, b = point_ids(ba, bb, v)
        pa.append(a)
        pb.append(b)
    pa, pb = np.array(pa, np.uint32), np.array(pb, np.uint32)
    vals = {m: orc.eval_pairs(F, m, pa, pb, k=K, bins=BINS) for m in range(4)}
    return ea, eb, pa, pb, vals


def test_graph_replay_matches_direct_launches(setup):
    F, boxes, pairs, runs = setup
    for a, b in zip(runs[True][1], runs[False][1]):
        for key in ("obs", "y", "mu", "var"):
            assert np.array_equal(a[key], b[key]), key
    assert runs[True][2] == runs[False][2]


def test_pool_and_observations(setup, orc):
    F, boxes, pairs, runs = setup
    _, states, res = runs[True]
    for rp, (pair, st) in enumerate(zip(pairs, states)):
        ea, eb = ext_of(boxes[pair[0]]), ext_of(boxes[pair[1]])
        assert np.array_equal(st["pool"], ogp.pool_positions(orc, SEED, rp, Q, ea, eb))
        assert len(st["obs"]) == R * T and len(set(st["obs"].tolist())) == R * T
        assert list(st["obs"][:R]) == list(range(R))
        _, _, pa, pb, vals = replay(orc, F, boxes, pair, rp, st)
        assert np.all(pa != pb)
        assert np.abs(st["y"] - vals[oracle.MI_KSG]).max() < 1e-5
        for m in range(4):  # running extremes over every evaluated sample
            assert abs(res[m][rp]["max"] - vals[m].max()) < 1e-5
            assert abs(res[m][rp]["min"] - vals[m].min()) < 1e-5
            assert res[m][rp]["count"] == R * T


def test_proposals_and_posterior(setup, orc):
    F, boxes, pairs, runs = setup
    _, states, _ = runs[True]
    for rp, (pair, st) in enumerate(zip(pairs, states)):
        ea, eb, pa, pb, vals = replay(orc, F, boxes, pair, rp, st)
        y = vals[oracle.MI_KSG]
        pool = st["pool"].astype(np.float64)
        m = float(np.mean(y[:R]))
        sf2 = max(float(np.mean((y[:R] - m) ** 2)), 1e-12)
        g = ogp.GP(0.25 * np.array(ea + eb, np.float64), sf2, 1e-4 * sf2)
        tol = 2e-3 * np.sqrt(sf2) + 1e-6
        for rnd in range(1, T):
            obs = st["obs"][:rnd * R]
            mu, var = g.posterior(pool[obs], y[:rnd * R], np.full(len(obs), m), pool,
                                  np.full(Q, m))
            ucb = mu + KAPPA * np.sqrt(np.maximum(var, 0))
            sel = np.zeros(Q, bool)
            sel[obs] = True
            sl = ogp.shortlist(ucb, sel, M)
            picks = list(st["obs"][rnd * R:(rnd + 1) * R])
            assert all(ucb[p] >= ucb[sl[-1]] - tol for p in picks), rnd  # in the shortlist
            # replay the greedy batch over the oracle's shortlist plus the GPU's picks
            # (a pick may sit at the shortlist boundary within fp32 noise)
            cand = np.array(list(sl) + [p for p in picks if p not in set(sl.tolist())])
            cov = g.posterior_cov(pool[obs], pool[cand])
            taken = np.zeros(len(cand), bool)
            for p in picks:  # each pick maximises the believer UCB (up to fp32 noise)
                i = int(np.nonzero(cand == p)[0][0])
                bu = mu[cand] + KAPPA * np.sqrt(np.maximum(np.diag(cov), 0))
                bu[taken] = -np.inf
                assert bu[i] >= bu.max() - tol, (rnd, p, bu[i], bu.max())
                taken[i] = True
                col = cov[:, i].copy()
                cov -= np.outer(col, col) / (col[i] + g.sn2)
        mu, var = g.posterior(pool[st["obs"]], y, np.full(R * T, m), pool, np.full(Q, m))
        assert np.abs(st["mu"] - mu).max() < 5e-3 * np.sqrt(sf2) + 1e-6
        assert np.abs(st["var"] - var).max() < 5e-3 * sf2 + 1e-9


@pytest.fixture(scope="module")
def setup2():
    """The same search over two variables on one grid (Section 4.3): the first
    point of a pair reads field A, the second field B."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03308_gb300 import Context, build
    build.build()
    Fa, Fb = gen.field(31, X, Y, Z, N), gen.field(32, X, Y, Z, N)
    ctx = Context(0)
    fa, fb = ctx.load_field(Fa), ctx.load_field(Fb)
    ra, rb = ctx.partition_regular(fa, 8, 8, 3), ctx.partition_regular(fb, 8, 8, 3)
    boxes = [ctx.region_info(r)[1] for r in ra]
    pairs = [(0, 7), (3, 3), (7, 0)]  # (3, 3): one brick, two variables, no self pair
    bos = ctx.bos_create(fa, [ra[a] for a, _ in pairs], [rb[b] for _, b in pairs], pool=Q,
                         per_round=R, rounds=T, shortlist=M, kappa=KAPPA, k=K, bins=BINS,
                         seed=SEED, field_b=fb)
    bos.run(T)
    yield Fa, Fb, boxes, pairs, [bos.inspect(i) for i in range(len(pairs))], bos.results()
    bos.close()
    ctx.close()


def test_two_field_observations(setup2, orc):
    Fa, Fb, boxes, pairs, states, res = setup2
    for rp, (pair, st) in enumerate(zip(pairs, states)):
        ba, bb = boxes[pair[0]], boxes[pair[1]]
        assert np.array_equal(st["pool"], ogp.pool_positions(orc, SEED, rp, Q, ext_of(ba),
                                                             ext_of(bb)))
        pa, pb = [], []
        for i, c in enumerate(st["obs"]):  # no self-pair fix: the variables differ
            v = ogp.bernoulli_voxels(orc, SEED, rp, i // R, i % R, st["pool"][c])
            a, b = point_ids(ba, bb, v)
            pa.append(a)
            pb.append(b)
        pa, pb = np.array(pa, np.uint32), np.array(pb, np.uint32)
        vals = {m: orc.eval_pairs(Fa, m, pa, pb, k=K, bins=BINS, Fb=Fb) for m in range(4)}
        assert np.abs(st["y"] - vals[oracle.MI_KSG]).max() < 1e-5
        for m in range(4):
            assert abs(res[m][rp]["max"] - vals[m].max()) < 1e-5
            assert abs(res[m][rp]["min"] - vals[m].min()) < 1e-5
            assert res[m][rp]["count"] == R * T


def test_two_field_matrix_is_asymmetric(setup2, orc):
    """Entries (A at brick 0, B at brick 7) and (A at brick 7, B at brick 0) are
    different searches: their maxima differ in general."""
    _, _, _, _, _, res = setup2
    assert res[oracle.PEARSON][0]["max"] != res[oracle.PEARSON][2]["max"]


def test_two_field_segment_extremes(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03308_gb300 import CC_MI_BINNED, CC_MI_KSG, CC_PEARSON, Context, Params
    Fa, Fb = gen.field(41, X, Y, Z, 60), gen.field(42, X, Y, Z, 60)
    ctx = Context(0)
    fa, fb = ctx.load_field(Fa), ctx.load_field(Fb)
    rng = np.random.default_rng(5)
    npts = X * Y * Z
    pa = rng.integers(0, npts, 5000).astype(np.uint32)
    pb = rng.integers(0, npts, 5000).astype(np.uint32)
    pb[:50] = pa[:50]  # the same voxel in both variables
    offs = [0, 1000, 1000, 3333, 5000]  # an empty segment, ragged sizes
    for kind in (CC_PEARSON, CC_MI_BINNED, CC_MI_KSG):
        ref = orc.eval_pairs(Fa, kind, pa, pb, k=5, bins=8, Fb=Fb)
        out = ctx.segment_extremes(fa, Params(kind, k=5, bins=8), pa, pb, offs, field_b=fb)
        for s in range(4):
            seg = ref[offs[s]:offs[s + 1]]
            assert out[s]["count"] == seg.size
            if seg.size:
                assert abs(out[s]["max"] - seg.max()) < 1e-5
                assert offs[s] <= out[s]["argmax"] < offs[s + 1]
                assert abs(ref[out[s]["argmax"]] - seg.max()) < 1e-5
                assert abs(out[s]["min"] - seg.min()) < 1e-5
    ctx.close()


LOCAL, LSCALE = 3, 0.0625


@pytest.fixture(scope="module")
def setup_local():
    """The batched search with LOCAL local proposals per round (from the second)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03308_gb300 import Context, build
    build.build()
    F = gen.field(31, X, Y, Z, N)
    ctx = Context(0)
    fid = ctx.load_field(F)
    rids = ctx.partition_regular(fid, 8, 8, 3)
    boxes = [ctx.region_info(r)[1] for r in rids]
    pairs = [(0, 7), (3, 3), (5, 20)]
    bos = ctx.bos_create(fid, [rids[a] for a, _ in pairs], [rids[b] for _, b in pairs], pool=Q,
                         per_round=R, rounds=T, shortlist=M, kappa=KAPPA, k=K, bins=BINS,
                         seed=SEED, local_picks=LOCAL, local_scale=LSCALE)
    bos.run(T)
    out = ([bos.inspect(i) for i in range(len(pairs))], [bos.samples(i) for i in range(len(pairs))],
           bos.results())
    yield (F, boxes, pairs) + out
    bos.close()
    ctx.close()


def test_local_proposals_against_oracle(setup_local, orc):
    """Every sample replayed through the oracle: round 0 takes the first R pool
    entries; later rounds start with LOCAL proposals around the two best
    samples so far (the oracle's incumbents of the replayed values, its FP64
    perturbation within fp32 rounding) followed by pool proposals, which alone
    are the GP's observations; rounding, values and running extremes exact."""
    F, boxes, pairs, states, samples, res = setup_local
    for rp, (pair, st, (theta, yall)) in enumerate(zip(pairs, states, samples)):
        ba, bb = boxes[pair[0]], boxes[pair[1]]
        ea, eb = ext_of(ba), ext_of(bb)
        ext = np.array(ea + eb, np.float64)
        pool = st["pool"]
        assert theta.shape == (R * T, 6) and yall.shape == (R * T,)
        assert np.array_equal(theta[:R], pool[:R])
        pa, pb = [], []
        for i in range(R * T):
            v = ogp.bernoulli_voxels(orc, SEED, rp, i // R, i % R, theta[i])
            if pair[0] == pair[1]:
                v = ogp.self_pair_fix(v, ea)
            a, b = point_ids(ba, bb, v)
            pa.append(a)
            pb.append(b)
        pa, pb = np.array(pa, np.uint32), np.array(pb, np.uint32)
        vals = {m: orc.eval_pairs(F, m, pa, pb, k=K, bins=BINS) for m in range(4)}
        assert np.abs(yall - vals[oracle.MI_KSG]).max() < 1e-5
        gp_obs = []
        for rnd in range(T):
            for j in range(R):
                i = rnd * R + j
                if rnd > 0 and j < LOCAL:
                    # incumbents among the samples before this round, on the GPU's values
                    inc = ogp.incumbents(theta[:rnd * R], list(yall[:rnd * R]))
                    want = ogp.local_theta(orc, SEED, rp, rnd, j, theta[inc[j % len(inc)]], ext,
                                           LSCALE)
                    assert np.abs(theta[i] - want).max() < 1e-4, (rnd, j, theta[i], want)
                else:
                    c = int(st["obs"][len(gp_obs)])
                    assert np.array_equal(theta[i], pool[c])
                    gp_obs.append(c)
        assert len(gp_obs) == len(st["obs"]) == R + (T - 1) * (R - LOCAL)
        assert np.abs(st["y"] - vals[oracle.MI_KSG][[i for i in range(R * T)
                                                     if i < R or i % R >= LOCAL]]).max() < 1e-5
        for m in range(4):  # running extremes over every sample, local ones included
            assert abs(res[m][rp]["max"] - vals[m].max()) < 1e-5
            assert abs(res[m][rp]["min"] - vals[m].min()) < 1e-5
            assert res[m][rp]["count"] == R * T
        # the GP posterior holds the pool observations only
        y = np.asarray(st["y"], np.float64)
        m0 = float(np.mean(y[:R]))
        sf2 = max(float(np.mean((y[:R] - m0) ** 2)), 1e-12)
        g = ogp.GP(0.25 * ext, sf2, 1e-4 * sf2)
        # every pool proposal of a round is a valid UCB / kriging-believer choice
        # of the posterior on the GP observations before that round
        tol = 2e-3 * np.sqrt(sf2) + 1e-6
        pool64 = pool.astype(np.float64)
        for rnd in range(1, T):
            s0 = R + (rnd - 1) * (R - LOCAL)
            obs = st["obs"][:s0]
            mu_r, var_r = g.posterior(pool64[obs], y[:s0], np.full(s0, m0), pool64,
                                      np.full(Q, m0))
            ucb = mu_r + KAPPA * np.sqrt(np.maximum(var_r, 0))
            sel = np.zeros(Q, bool)
            sel[obs] = True
            sl = ogp.shortlist(ucb, sel, M)
            picks = list(st["obs"][s0:s0 + R - LOCAL])
            assert all(ucb[p] >= ucb[sl[-1]] - tol for p in picks), rnd
            cand = np.array(list(sl) + [p for p in picks if p not in set(sl.tolist())])
            cov = g.posterior_cov(pool64[obs], pool64[cand])
            taken = np.zeros(len(cand), bool)
            for p in picks:
                i = int(np.nonzero(cand == p)[0][0])
                bu = mu_r[cand] + KAPPA * np.sqrt(np.maximum(np.diag(cov), 0))
                bu[taken] = -np.inf
                assert bu[i] >= bu.max() - tol, (rnd, p, bu[i], bu.max())
                taken[i] = True
                col = cov[:, i].copy()
                cov -= np.outer(col, col) / (col[i] + g.sn2)
        mu, var = g.posterior(pool64[st["obs"]], y, np.full(len(y), m0), pool64,
                              np.full(Q, m0))
        assert np.abs(st["mu"] - mu).max() < 5e-3 * np.sqrt(sf2) + 1e-6
        assert np.abs(st["var"] - var).max() < 5e-3 * sf2 + 1e-9


def test_local_picks_argument_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03308_gb300 import CCError, Context
    F = gen.field(31, X, Y, Z, N)
    ctx = Context(0)
    fid = ctx.load_field(F)
    rids = ctx.partition_regular(fid, 8, 8, 3)
    for kw in (dict(local_picks=R), dict(local_picks=-1), dict(local_picks=2, local_scale=0.0)):
        with pytest.raises(CCError):
            ctx.bos_create(fid, [rids[0]], [rids[1]], pool=Q, per_round=R, rounds=T, shortlist=M,
                           **kw)
    ctx.close()
