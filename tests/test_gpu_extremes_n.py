"""Member counts at the edges of every code path, against the FP64 oracle:
n = 2 (the smallest ensemble), 3, 31 / 32 / 33 (one lane slice and the
smallest sample-stream KSG), 255 / 256 / 257 (the largest stream KSG, the
integer-rank BF16 limit), 1023 / 1024 (the largest ensemble). Every measure
on pair batches (ranks, bins and KSG counts bit-exact), FP32 all-pairs and the
certified BF16 path with a sorted top list."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
TOL = 1e-5
NS = [2, 3, 31, 32, 33, 255, 256, 257, 1023, 1024]


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03308_gb300 import Context, build
    build.build()
    ctx = Context(0)
    yield ctx
    ctx.close()


@pytest.mark.parametrize("n", NS)
def test_pair_measures_at_member_count(cc, orc, n):
    from paper_2309_03308_gb300 import Params
    X, Y, Z = 9, 7, 2  # 126 points
    F = gen.field(70 + n, X, Y, Z, n)
    F[:, 0, 0, 3] = 0.25  # a constant member vector (zero variance)
    fid = cc.load_field(F)
    P = X * Y * Z
    i, j = np.triu_indices(P, 1)
    step = 1 if n <= 257 else 23  # bounded oracle time at n ~ 1000
    pa, pb = i[::step].astype(np.uint32), j[::step].astype(np.uint32)
    k = min(3, n - 1)
    for kind, kw in ((oracle.PEARSON, {}), (oracle.SPEARMAN, {}),
                     (oracle.MI_BINNED, {"bins": 8}), (oracle.MI_KSG, {"k": k})):
        got = cc.eval_pairs(fid, fid, Params(kind, **kw), pa, pb)
        ref = orc.eval_pairs(F, kind, pa, pb, **kw)
        assert np.abs(got - ref).max() < TOL, (n, kind)
    _, nx, ny, eps = cc.ksg_counts(fid, fid, k, pa[:200], pb[:200], n)
    _, rx, ry, reps = orc.eval_pairs(F, oracle.MI_KSG, pa[:200], pb[:200], k=k, want_ksg=True)
    assert np.array_equal(nx, rx) and np.array_equal(ny, ry) and np.array_equal(eps, reps)
    pts = np.arange(P, dtype=np.uint32)
    assert np.array_equal(cc.get_plane(fid, 0, pts, n), orc.rank2(F, pts))
    assert np.array_equal(cc.get_plane(fid, 1, pts, n, bins=8), orc.bins(F, pts, 8))
    cc.free_field(fid)


@pytest.mark.parametrize("n", [2, 33, 257, 1024])
def test_all_pairs_at_member_count(cc, orc, n):
    from paper_2309_03308_gb300 import CC_BF16, CC_PEARSON, CC_SPEARMAN, Params
    X, Y, Z = 40, 20, 2  # regions of 20 x 20 x 2 = 800 points
    F = gen.field(90 + n, X, Y, Z, n)
    fid = cc.load_field(F)
    ra, rb = cc.define_regions(fid, [(0, 0, 0, 20, 20, 2), (20, 0, 0, 40, 20, 2)])
    A = oracle.box_points(X, Y, Z, (0, 0, 0, 20, 20, 2))
    B = oracle.box_points(X, Y, Z, (20, 0, 0, 40, 20, 2))
    for kind in (CC_PEARSON, CC_SPEARMAN):
        ref = orc.region_extremes(F, A, B, False, kind)
        res = cc.all_pairs(ra, rb, Params(kind))
        assert res["count"] == ref["count"] == 640000
        assert abs(res["max"] - ref["max"]) < TOL and abs(res["min"] - ref["min"]) < TOL
        res, ids, vals, cert = cc.all_pairs_topk(ra, rb, Params(kind, precision=CC_BF16),
                                                 topk=64)
        assert cert["certified_max"] == 1 and cert["certified_min"] == 1
        assert abs(res["max"] - ref["max"]) < 1e-6 and abs(res["min"] - ref["min"]) < 1e-6
        assert np.all(np.diff(vals) <= 0) and vals[0] == res["max"]
        a, b = ids // 800, ids % 800
        exact = orc.eval_pairs(F, kind, A[a].astype(np.uint32), B[b].astype(np.uint32))
        assert np.abs(exact - vals).max() < 1e-6
    cc.free_field(fid)
