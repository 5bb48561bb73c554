"""All pairs between two regions (FP32 SIMT tiles, fused extremes) against the
FP64 oracle: every region pair of the small config, ragged tiles, full-size
focus regions on sampled outputs."""
import numpy as np
import pytest

import gen
import oracle
from gen import configs

pytestmark = pytest.mark.gpu
TOL = 1e-5


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


def check_extremes(res, ref, vals=None):
    assert res["count"] == ref["count"]
    assert abs(res["max"] - ref["max"]) < TOL and abs(res["min"] - ref["min"]) < TOL
    if vals is not None:  # the reported argmax/argmin are valid maximisers/minimisers
        assert abs(vals[res["argmax"]] - ref["max"]) < TOL
        assert abs(vals[res["argmin"]] - ref["min"]) < TOL


@pytest.mark.parametrize("kind", [oracle.PEARSON, oracle.SPEARMAN], ids=["pearson", "spearman"])
def test_small_region_pairs(cc, orc, kind):
    from paper_2309_03308_gb300 import Params
    c = configs.SMALL
    F = gen.field(c["seed"], c["X"], c["Y"], c["Z"], c["n"])
    fid = cc.load_field(F)
    rids = cc.partition_regular(fid, *c["region"])
    boxes = configs.regular_boxes(c["X"], c["Y"], c["Z"], *c["region"])
    assert len(rids) == 8 and [cc.region_info(r)[1] for r in rids] == boxes
    total = 0
    for i in range(8):
        for j in range(i, 8):
            A = oracle.box_points(c["X"], c["Y"], c["Z"], boxes[i])
            B = oracle.box_points(c["X"], c["Y"], c["Z"], boxes[j])
            ref = orc.region_extremes(F, A, B, i == j, kind, want_values=True)
            res = cc.all_pairs(rids[i], rids[j], Params(kind))
            check_extremes(res, ref, ref["values"])
            total += res["count"]
    assert total == 523776


def test_values_store_and_ragged_tiles(cc, orc):
    import torch
    from paper_2309_03308_gb300 import Params
    X, Y, Z, n = 23, 19, 5, 40
    F = gen.field(9, X, Y, Z, n)
    fid = cc.load_field(F)
    boxes = [(1, 2, 0, 8, 11, 3), (10, 3, 1, 23, 8, 5)]  # 189 and 260 points
    ra, rb = cc.define_regions(fid, boxes)
    A = oracle.box_points(X, Y, Z, boxes[0])
    B = oracle.box_points(X, Y, Z, boxes[1])
    for kind in (oracle.PEARSON, oracle.SPEARMAN):
        for (r1, r2, P1, P2) in ((ra, rb, A, B), (rb, rb, B, B), (rb, ra, B, A)):
            ld = len(P2) + 3  # odd leading dimension: scalar stores
            vals = torch.full((len(P1), ld), 7.0, device="cuda")
            res = cc.all_pairs(r1, r2, Params(kind), values=vals, ld=ld)
            got = vals.cpu().numpy()
            ref = orc.region_extremes(F, P1, P2, r1 == r2, kind, want_values=True)
            full = orc.eval_pairs(F, kind, np.repeat(P1, len(P2)), np.tile(P2, len(P1)))
            assert np.abs(got[:, :len(P2)] - full.reshape(len(P1), len(P2))).max() < TOL
            assert np.all(got[:, len(P2):] == 7.0)  # padding columns untouched
            check_extremes(res, ref, ref["values"])


def test_inter_field_regions(cc, orc):
    from paper_2309_03308_gb300 import Params
    F1 = gen.field(21, 10, 9, 3, 24)
    F2 = gen.field(22, 10, 9, 3, 24)
    f1, f2 = cc.load_field(F1), cc.load_field(F2)
    (r1,) = cc.define_regions(f1, [(0, 0, 0, 10, 9, 3)])
    (r2,) = cc.define_regions(f2, [(0, 0, 0, 10, 9, 3)])
    res = cc.all_pairs(r1, r2, Params(oracle.PEARSON))
    P = np.arange(270, dtype=np.uint32)
    full = orc.eval_pairs(F1, oracle.PEARSON, np.repeat(P, 270), np.tile(P, 270), Fb=F2)
    assert res["count"] == 270 * 270
    assert abs(res["max"] - full.max()) < TOL and abs(full[res["argmax"]] - full.max()) < TOL


def test_focus_full_size_sampled(cc, orc):
    import torch
    from paper_2309_03308_gb300 import Params
    c = configs.FOCUS
    F = gen.field(c["seed"], c["X"], c["Y"], c["Z"], c["n"])
    fid = cc.load_field(F)
    ra, rb = cc.define_regions(fid, [c["box_a"], c["box_b"]])
    A = oracle.box_points(c["X"], c["Y"], c["Z"], c["box_a"])
    B = oracle.box_points(c["X"], c["Y"], c["Z"], c["box_b"])
    vals = torch.empty((len(A), len(B)), device="cuda")
    rng = np.random.default_rng(8)
    ia = rng.integers(0, len(A), 100000)
    ib = rng.integers(0, len(B), 100000)
    for kind in (oracle.PEARSON, oracle.SPEARMAN):
        res = cc.all_pairs(ra, rb, Params(kind), values=vals)
        assert res["count"] == 20480 * 20480
        got = vals[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
        ref = orc.eval_pairs(F, kind, A[ia], B[ib])
        assert np.abs(got - ref).max() < TOL
        # reported extremes are attained by the reported pairs and bound the sample
        a, b = divmod(res["argmax"], len(B))
        a2, b2 = divmod(res["argmin"], len(B))
        e = orc.eval_pairs(F, kind, np.array([A[a], A[a2]]), np.array([B[b], B[b2]]))
        assert abs(e[0] - res["max"]) < TOL and abs(e[1] - res["min"]) < TOL
        assert res["max"] >= ref.max() - TOL and res["min"] <= ref.min() + TOL
        # the stored matrix agrees with the fused reduction
        assert abs(vals.max().item() - res["max"]) < 1e-7
