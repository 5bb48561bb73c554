"""Reduced-precision all-pairs (BF16 / FP8 E4M3 tensor-core contraction) with
Dot2 re-evaluation and certified extremes, against the FP64 oracle on every
pair. Refined values are compensated fp32 products of the fp32 planes, so they
are held to 1e-6 of the exact correlation."""
import numpy as np
import pytest

import gen
import oracle
from gen import configs

pytestmark = pytest.mark.gpu
TOL_REFINED = 1e-6


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


def two_fields(n, box_a, box_b, seed=2):
    Fa = gen.field(seed, 352, 256, 20, n, box=box_a)
    Fb = gen.field(seed, 352, 256, 20, n, box=box_b)
    return Fa, Fb


def all_values(orc, kind, Fa, Fb):
    na, nb = Fa[0].size, Fb[0].size
    A = np.arange(na, dtype=np.uint32)
    B = np.arange(nb, dtype=np.uint32)
    return orc.eval_pairs(Fa, kind, np.repeat(A, nb), np.tile(B, na), Fb=Fb)


def check(res, ids, vals, cert, full, count, topk):
    assert res["count"] == count
    assert cert["certified_max"] == 1 and cert["certified_min"] == 1, cert
    assert abs(res["max"] - full.max()) < TOL_REFINED, (res["max"], full.max())
    assert abs(res["min"] - full.min()) < TOL_REFINED, (res["min"], full.min())
    assert abs(full[res["argmax"]] - full.max()) < TOL_REFINED
    assert abs(full[res["argmin"]] - full.min()) < TOL_REFINED
    if topk:
        assert np.all(np.diff(vals) <= 0) and vals[0] == res["max"]
        assert np.all(ids < full.size)
        assert np.abs(full[ids.astype(np.int64)] - vals).max() < TOL_REFINED
        kth = np.sort(full)[::-1][topk - 1]
        assert vals[-1] >= kth - 2 * cert["bound"]


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_pearson_n1000_cross_ragged(cc, orc, prec):
    from paper_2309_03308_gb300 import CC_BF16, CC_FP8_E4M3, CC_PEARSON, Params
    p = {"bf16": CC_BF16, "fp8": CC_FP8_E4M3}[prec]
    Fa, Fb = two_fields(1000, (64, 64, 0, 89, 74, 4), (256, 160, 0, 291, 180, 1))  # 1000 x 700
    fa, fb = cc.load_field(Fa), cc.load_field(Fb)
    (ra,) = cc.define_regions(fa, [(0, 0, 0, 25, 10, 4)])
    (rb,) = cc.define_regions(fb, [(0, 0, 0, 35, 20, 1)])
    full = all_values(orc, oracle.PEARSON, Fa, Fb)
    res, ids, vals, cert = cc.all_pairs_topk(ra, rb, Params(CC_PEARSON, precision=p), topk=64)
    check(res, ids, vals, cert, full, 1000 * 700, 64)
    assert cert["bound"] < (0.02 if prec == "bf16" else 0.2)


def test_self_pair_bf16(cc, orc):
    from paper_2309_03308_gb300 import CC_BF16, CC_PEARSON, Params
    Fa = gen.field(2, 352, 256, 20, 1000, box=(100, 100, 0, 132, 116, 2))  # 1024 points
    fa = cc.load_field(Fa)
    (ra,) = cc.define_regions(fa, [(0, 0, 0, 32, 16, 2)])
    res, ids, vals, cert = cc.all_pairs_topk(ra, ra, Params(CC_PEARSON, precision=CC_BF16),
                                             topk=100)
    full = all_values(orc, oracle.PEARSON, Fa, Fa).reshape(1024, 1024)
    mask = np.triu(np.ones((1024, 1024), bool), 1)
    full = np.where(mask, full, np.nan).ravel()
    valid = full[~np.isnan(full)]
    assert res["count"] == 1024 * 1023 // 2
    assert cert["certified_max"] == 1 and cert["certified_min"] == 1
    assert abs(res["max"] - valid.max()) < TOL_REFINED
    assert abs(res["min"] - valid.min()) < TOL_REFINED
    a, b = divmod(res["argmax"], 1024)
    assert a < b
    assert np.abs(full[ids.astype(np.int64)] - vals).max() < TOL_REFINED


@pytest.mark.parametrize("n", [32, 100, 257])
def test_spearman_bf16_integer_ranks_exact(cc, orc, n):
    """n <= 257: the BF16 contraction of integer centred ranks is exact, so the
    certificate bound is only the epilogue's fp32 scaling (~1e-6) and the
    refined extremes and top list match the FP64 Spearman values, with ties."""
    from paper_2309_03308_gb300 import CC_BF16, CC_SPEARMAN, Params
    Fa, Fb = two_fields(n, (64, 64, 0, 96, 80, 2), (256, 160, 0, 280, 176, 1))  # 1024 x 384
    Fa = np.round(Fa * 2) / 2  # heavy ties: average ranks, odd doubled ranks
    fa, fb = cc.load_field(Fa.astype(np.float32)), cc.load_field(Fb)
    (ra,) = cc.define_regions(fa, [(0, 0, 0, 32, 16, 2)])
    (rb,) = cc.define_regions(fb, [(0, 0, 0, 24, 16, 1)])
    full = all_values(orc, oracle.SPEARMAN, Fa.astype(np.float32), Fb)
    res, ids, vals, cert = cc.all_pairs_topk(ra, rb, Params(CC_SPEARMAN, precision=CC_BF16),
                                             topk=512)
    assert cert["bound"] < 2e-6, cert
    check(res, ids, vals, cert, full, full.size, 512)
    cc.free_field(fa)
    cc.free_field(fb)


def test_spearman_n100_and_cc_all_pairs_route(cc, orc):
    from paper_2309_03308_gb300 import CC_BF16, CC_FP8_E4M3, CC_SPEARMAN, Params
    Fa, Fb = two_fields(100, (64, 64, 0, 96, 96, 2), (256, 160, 0, 288, 176, 1))  # 2048 x 512
    fa, fb = cc.load_field(Fa), cc.load_field(Fb)
    (ra,) = cc.define_regions(fa, [(0, 0, 0, 32, 32, 2)])
    (rb,) = cc.define_regions(fb, [(0, 0, 0, 32, 16, 1)])
    full = all_values(orc, oracle.SPEARMAN, Fa, Fb)
    for p in (CC_BF16, CC_FP8_E4M3):
        res = cc.all_pairs(ra, rb, Params(CC_SPEARMAN, precision=p))
        assert abs(res["max"] - full.max()) < TOL_REFINED
        assert abs(res["min"] - full.min()) < TOL_REFINED
        assert abs(full[res["argmax"]] - full.max()) < TOL_REFINED


def test_dot2_pairs_n1000(cc, orc):
    from paper_2309_03308_gb300 import CC_FP32, CC_FP32_DOT2, CC_PEARSON, CC_SPEARMAN, Params
    F = gen.field(2, 352, 256, 20, 1000, box=(10, 10, 0, 42, 42, 1))
    fid = cc.load_field(F)
    rng = np.random.default_rng(3)
    pa = rng.integers(0, 1024, 3000).astype(np.uint32)
    pb = rng.integers(0, 1024, 3000).astype(np.uint32)
    for kind in (CC_PEARSON, CC_SPEARMAN):
        ref = orc.eval_pairs(F, kind, pa, pb)
        d2 = cc.eval_pairs(fid, fid, Params(kind, precision=CC_FP32_DOT2), pa, pb)
        f32 = cc.eval_pairs(fid, fid, Params(kind, precision=CC_FP32), pa, pb)
        assert np.abs(d2 - ref).max() < TOL_REFINED
        assert np.abs(d2 - ref).max() <= np.abs(f32 - ref).max() + 1e-7


def test_mixed_argument_errors(cc):
    from paper_2309_03308_gb300 import CC_BF16, CC_MI_KSG, CC_PEARSON, CCError, Params
    F = gen.field(3, 8, 8, 2, 40)
    fid = cc.load_field(F)
    (r,) = cc.define_regions(fid, [(0, 0, 0, 8, 8, 2)])
    with pytest.raises(CCError):
        cc.all_pairs_topk(r, r, Params(CC_PEARSON, precision=CC_BF16), topk=5000)
    with pytest.raises(CCError):
        cc.all_pairs_topk(r, r, Params(CC_MI_KSG, precision=CC_BF16))
    with pytest.raises(CCError):
        cc.all_pairs_topk(r, r, Params(CC_PEARSON))  # FP32 is not a reduced precision


def chunk_extremes(full, na, nb):
    """Per (32-column chunk, row) max and min of an [na][nb] value matrix, [chunks][na]."""
    chunks = (nb + 31) // 32
    pad = np.full((na, chunks * 32), np.nan)
    pad[:, :nb] = full.reshape(na, nb)
    v = pad.reshape(na, chunks, 32)
    return np.nanmax(v, 2).T, np.nanmin(v, 2).T


APPROX_CASES = [  # (n, box of field A, box of field B, region A, region B): |A| x |B|
    (1000, (64, 64, 0, 89, 74, 4), (256, 160, 0, 291, 180, 1), (0, 0, 0, 25, 10, 4),
     (0, 0, 0, 35, 20, 1)),                                                   # 1000 x 700
    (100, (64, 64, 0, 96, 96, 2), (256, 160, 0, 288, 176, 1), (0, 0, 0, 32, 32, 2),
     (0, 0, 0, 32, 16, 1)),                                                   # 2048 x 512
]


@pytest.mark.parametrize("case", range(len(APPROX_CASES)), ids=["n1000_1000x700", "n100_2048x512"])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_approx_values_within_stated_bound(cc, orc, case, prec):
    """Every approximate chunk extreme of the tensor-core contraction lies within
    the certified bound of the FP64 oracle's chunk extreme (the bound is stated
    for the fp32 planes; their own rounding adds < 1e-6)."""
    from paper_2309_03308_gb300 import CC_BF16, CC_FP8_E4M3, CC_PEARSON, Params
    p = {"bf16": CC_BF16, "fp8": CC_FP8_E4M3}[prec]
    n, bxa, bxb, rga, rgb = APPROX_CASES[case]
    Fa, Fb = two_fields(n, bxa, bxb)
    fa, fb = cc.load_field(Fa), cc.load_field(Fb)
    (ra,) = cc.define_regions(fa, [rga])
    (rb,) = cc.define_regions(fb, [rgb])
    na, nb = Fa[0].size, Fb[0].size
    full = all_values(orc, oracle.PEARSON, Fa, Fb)
    cmax, cmin, bound = cc.all_pairs_approx(ra, rb, Params(CC_PEARSON, precision=p))
    emax, emin = chunk_extremes(full, na, nb)
    err = np.maximum(np.abs(cmax - emax), np.abs(cmin - emin))
    print(f"n={n} {prec}: observed max {err.max():.3e} mean {err.mean():.3e} bound {bound:.3e}")
    assert err.max() <= bound + 1e-6, (err.max(), bound)
    # the bound is the one the certified path uses, and is not vacuous
    _, _, _, cert = cc.all_pairs_topk(ra, rb, Params(CC_PEARSON, precision=p), topk=0)
    assert abs(cert["bound"] - bound) <= 1e-6 * bound
    assert bound < (0.02 if prec == "bf16" else 0.2)
    cc.free_field(fa)
    cc.free_field(fb)


def test_approx_self_pair_masks_excluded_pairs(cc, orc):
    """A self region pair: chunk entries with no pair b > a are -inf / +inf and
    the rest lie within the bound of the oracle's extremes over b > a."""
    from paper_2309_03308_gb300 import CC_BF16, CC_PEARSON, Params
    Fa = gen.field(2, 352, 256, 20, 100, box=(100, 100, 0, 132, 116, 2))  # 1024 points
    fa = cc.load_field(Fa)
    (ra,) = cc.define_regions(fa, [(0, 0, 0, 32, 16, 2)])
    full = all_values(orc, oracle.PEARSON, Fa, Fa).reshape(1024, 1024)
    full = np.where(np.triu(np.ones((1024, 1024), bool), 1), full, np.nan)
    cmax, cmin, bound = cc.all_pairs_approx(ra, ra, Params(CC_PEARSON, precision=CC_BF16))
    with np.errstate(all="ignore"):
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", RuntimeWarning)
            emax, emin = chunk_extremes(full.ravel(), 1024, 1024)
    empty = np.isnan(emax)
    assert np.all(cmax[empty] == -np.inf) and np.all(cmin[empty] == np.inf)
    assert np.abs(cmax[~empty] - emax[~empty]).max() <= bound + 1e-6
    assert np.abs(cmin[~empty] - emin[~empty]).max() <= bound + 1e-6
    cc.free_field(fa)


def test_focus_full_size_bf16_certified_against_oracle(cc, orc):
    """The certified BF16 path on the full 20,480 x 20,480 focus region pair:
    the reported maximum, minimum and the sorted top 4096 are exact FP64 values
    of the reported pairs (within the compensated-fp32 tolerance), and no pair
    of a 100,000-pair uniform sample exceeds them."""
    from paper_2309_03308_gb300 import CC_BF16, CC_PEARSON, Params
    c = configs.FOCUS
    F = gen.field(c["seed"], c["X"], c["Y"], c["Z"], c["n"])
    fid = cc.load_field(F)
    ra, rb = cc.define_regions(fid, [c["box_a"], c["box_b"]])
    A = oracle.box_points(c["X"], c["Y"], c["Z"], c["box_a"])
    B = oracle.box_points(c["X"], c["Y"], c["Z"], c["box_b"])
    res, ids, vals, cert = cc.all_pairs_topk(ra, rb, Params(CC_PEARSON, precision=CC_BF16),
                                             topk=4096)
    assert cert["certified_max"] == 1 and cert["certified_min"] == 1, cert
    assert res["count"] == len(A) * len(B)
    ia, ib = np.divmod(ids.astype(np.int64), len(B))
    top = orc.eval_pairs(F, oracle.PEARSON, A[ia], B[ib])
    assert np.abs(top - vals).max() < TOL_REFINED
    assert np.all(np.diff(vals) <= 0) and vals[0] == res["max"]
    a, b = divmod(res["argmax"], len(B))
    a2, b2 = divmod(res["argmin"], len(B))
    e = orc.eval_pairs(F, oracle.PEARSON, np.array([A[a], A[a2]]), np.array([B[b], B[b2]]))
    assert abs(e[0] - res["max"]) < TOL_REFINED and abs(e[1] - res["min"]) < TOL_REFINED
    rng = np.random.default_rng(12)
    sa = rng.integers(0, len(A), 100000)
    sb = rng.integers(0, len(B), 100000)
    ref = orc.eval_pairs(F, oracle.PEARSON, A[sa], B[sb])
    assert ref.max() <= res["max"] + TOL_REFINED and ref.min() >= res["min"] - TOL_REFINED
    # sampled pairs above the list's last value are in the list
    above = ref > vals[-1] + 2 * cert["bound"]
    listed = set((ia * len(B) + ib).tolist())
    assert all(int(x) in listed for x in (sa[above] * len(B) + sb[above]))
    cc.free_field(fid)


def test_partial_row_tile_after_larger_call(cc, orc):
    """A region of 100 points pads to 256 rows, two row tiles of 128 of which
    only the first holds real points. Every padded row's chunk extremes must be
    written by the call itself: here an earlier call on 256 points that
    include the column region (so its extremes reach 1) used the same scratch
    layout just before, and a stale row left in place would take candidate
    slots from the real chunks. The second call's extremes, certificate and
    top list are checked against the FP64 oracle."""
    from paper_2309_03308_gb300 import CC_BF16, CC_PEARSON, Params
    F = gen.field(2, 352, 256, 20, 100, box=(64, 64, 0, 96, 96, 20))  # 32 x 32 x 20 points
    fid = cc.load_field(F)
    rb, rbig, rsmall = cc.define_regions(
        fid, [(0, 0, 0, 32, 32, 20), (0, 0, 0, 16, 16, 1), (20, 20, 10, 30, 30, 11)])
    prm = Params(CC_PEARSON, precision=CC_BF16)
    res0, _, _, cert0 = cc.all_pairs_topk(rbig, rb, prm, topk=4096)
    assert res0["max"] > 0.999 and cert0["certified_max"] == 1  # a point paired with itself
    res, ids, vals, cert = cc.all_pairs_topk(rsmall, rb, prm, topk=4096)
    full = all_values(orc, oracle.PEARSON, np.ascontiguousarray(F[:, 10:11, 20:30, 20:30]), F)
    check(res, ids, vals, cert, full, 100 * 20480, 4096)
    assert np.all(ids < full.size)  # every listed pair has a real row
    cc.free_field(fid)
