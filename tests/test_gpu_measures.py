"""CUDA path against the FP64 oracle through the C ABI (pair batches, planes,
sampler, segment extremes). Tolerances: 1e-5 absolute for fp32 correlation
values and MI; ranks, bins and KSG neighbour counts bit-exact."""
import math

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


@pytest.fixture(scope="module")
def small(cc):
    c = configs.SMALL
    F = gen.field(c["seed"], c["X"], c["Y"], c["Z"], c["n"])
    fid = cc.load_field(F)
    return F, fid


@pytest.fixture(scope="module")
def focus(cc):
    c = configs.FOCUS
    F = gen.field(c["seed"], c["X"], c["Y"], c["Z"], c["n"])
    fid = cc.load_field(F)
    ra, rb = cc.define_regions(fid, [c["box_a"], c["box_b"]])
    return F, fid, ra, rb


def all_unique_pairs(P):
    i, j = np.triu_indices(P, 1)
    return i.astype(np.uint32), j.astype(np.uint32)


# ---------------------------------------------------------------- planes (bit-exact)
def test_planes_bit_exact(cc, small, orc):
    F, fid = small
    n = F.shape[0]
    pts = np.arange(F[0].size, dtype=np.uint32)
    assert np.array_equal(cc.get_plane(fid, 0, pts, n), orc.rank2(F, pts))
    for B in (8, 16):
        assert np.array_equal(cc.get_plane(fid, 1, pts, n, bins=B), orc.bins(F, pts, B))
    srt = cc.get_plane(fid, 2, pts, n)
    assert np.array_equal(srt, np.sort(F.reshape(n, -1).T, axis=1))


def test_planes_with_ties(cc, orc):
    rng = np.random.default_rng(3)
    F = rng.integers(-3, 4, (40, 3, 4, 5)).astype(np.float32)
    F[:, 0, 0, 0] = 1.5  # constant member vector
    F[5, 1, 1, 1] = -0.0
    F[6, 1, 1, 1] = 0.0
    fid = cc.load_field(F)
    pts = np.arange(60, dtype=np.uint32)
    assert np.array_equal(cc.get_plane(fid, 0, pts, 40), orc.rank2(F, pts))
    for B in (2, 5, 16):
        assert np.array_equal(cc.get_plane(fid, 1, pts, 40, bins=B), orc.bins(F, pts, B))
    z = cc.get_plane(fid, 3, pts[:1], 40)
    assert np.all(z == 0)


def _near_equal_rows(n, rng):
    """Member vectors whose values sit a fixed number of ulps apart (1, 127,
    128, 129) around 1 and -1, subnormals around zero with both signed zeros,
    one 1-ulp pair in random data, and random rows, each row permuted."""
    one = np.float32(1.0).view(np.int32)
    rows = []
    for step in (1, 127, 128, 129):
        rows.append((one + step * np.arange(n, dtype=np.int32)).view(np.float32))
    rows.append(-(one + np.arange(n, dtype=np.int32)).view(np.float32))
    sub = (np.arange(n, dtype=np.int32) - n // 2).astype(np.float32) * np.float32(2.0 ** -149)
    sub[0], sub[1] = np.float32(-0.0), np.float32(0.0)
    rows.append(sub)
    r = rng.standard_normal(n).astype(np.float32)
    r[1] = (r[0].view(np.int32) + 1).view(np.float32)
    rows.append(r)
    for _ in range(9):
        rows.append(rng.standard_normal(n).astype(np.float32))
    return np.stack([rng.permutation(x) for x in rows], axis=1)  # [n][rows]


@pytest.mark.parametrize("n", [32, 100, 128])
def test_planes_near_equal_values(cc, orc, n):
    """Values closer than the sort's first-pass key resolution (2^7 ulp), but
    distinct, next to rows that it separates: ranks, sorted values and bins
    bit-exact, z-scores within a few fp32 roundings, KSG counts bit-exact."""
    rng = np.random.default_rng(17 + n)
    F = _near_equal_rows(n, rng).reshape(n, 1, 4, 4)
    fid = cc.load_field(F)
    pts = np.arange(16, dtype=np.uint32)
    assert np.array_equal(cc.get_plane(fid, 0, pts, n), orc.rank2(F, pts))
    for B in (8, 16):
        assert np.array_equal(cc.get_plane(fid, 1, pts, n, bins=B), orc.bins(F, pts, B))
    srt = cc.get_plane(fid, 2, pts, n)
    assert np.array_equal(srt, np.sort(F.reshape(n, -1).T, axis=1))
    z = cc.get_plane(fid, 3, pts, n).astype(np.float64)
    V = F.reshape(n, -1).T.astype(np.float64)
    d = V - V.mean(axis=1, keepdims=True)
    ss = (d * d).sum(axis=1, keepdims=True)
    ref = np.divide(d, np.sqrt(ss), out=np.zeros_like(d), where=ss > 0)
    assert np.all(np.abs(z - ref) <= 4 * 2.0 ** -24 * np.abs(ref).max(axis=1, keepdims=True))
    pa, pb = np.meshgrid(pts, pts, indexing="ij")
    pa, pb = pa.ravel(), pb.ravel()
    out, nx, ny, eps = cc.ksg_counts(fid, fid, 3, pa, pb, n)
    ref_v, rnx, rny, reps = orc.eval_pairs(F, oracle.MI_KSG, pa, pb, k=3, want_ksg=True)
    assert np.array_equal(eps, reps)
    assert np.array_equal(nx, rnx) and np.array_equal(ny, rny)
    cc.free_field(fid)


def test_update_field_rebuilds_every_plane(cc, orc):
    """After cc_update_field the planes, including the bin planes of the bin
    counts already in use (rebuilt in the per-point pass) and of a new bin
    count (built lazily), equal the oracle's for the new values."""
    import torch
    from paper_2309_03308_gb300 import CC_MI_BINNED, Params
    X, Y, Z, n = 12, 10, 3, 100
    F1 = gen.field(31, X, Y, Z, n)
    F2 = gen.field(32, X, Y, Z, n)
    F2[:, 0, 0, 0] = 2.5  # a constant member vector
    fid = cc.load_field(F1)
    pts = np.arange(X * Y * Z, dtype=np.uint32)
    for B in (8, 16):
        cc.get_plane(fid, 1, pts[:4], n, bins=B)  # bins for 8 and 16 are now in use
    for src in (F2, torch.from_numpy(F2).cuda()):
        cc.update_field(fid, src)
        for B in (8, 16, 5):
            assert np.array_equal(cc.get_plane(fid, 1, pts, n, bins=B), orc.bins(F2, pts, B)), B
        assert np.array_equal(cc.get_plane(fid, 0, pts, n), orc.rank2(F2, pts))
        srt = cc.get_plane(fid, 2, pts, n)
        assert np.array_equal(srt, np.sort(F2.reshape(n, -1)[:, pts].T, axis=1))
        pa, pb = all_unique_pairs(X * Y * Z)
        pa, pb = pa[::37].copy(), pb[::37].copy()
        for B in (8, 16):
            got = cc.eval_pairs(fid, fid, Params(CC_MI_BINNED, bins=B), pa, pb)
            ref = orc.eval_pairs(F2, oracle.MI_BINNED, pa, pb, bins=B)
            assert np.abs(got - ref).max() < TOL
    cc.free_field(fid)


def test_update_from_host_in_overlapped_chunks(cc):
    """A host-data update above 64 MB is copied and ingested in point ranges
    on two streams: every plane equals that of the same values loaded from
    device memory in one pass (bit for bit), including the bin planes rebuilt
    in the per-point pass and the ragged last range."""
    import torch
    from paper_2309_03308_gb300 import CC_PLANE_BINS, CC_PLANE_RANK2, CC_PLANE_SORTED, CC_PLANE_ZHAT
    X, Y, Z, n = 131, 67, 20, 100  # 175,540 points (not a multiple of 8), 70 MB
    F1 = gen.field(41, X, Y, Z, n)
    F2 = gen.field(42, X, Y, Z, n)
    upd = cc.load_field(F1)
    ref = cc.load_field(torch.from_numpy(F2).cuda())
    pts = np.arange(0, X * Y * Z, 7, dtype=np.uint32)
    for f in (upd, ref):
        cc.get_plane(f, CC_PLANE_BINS, pts[:4], n, bins=16)  # 16-bin planes in use
    for _ in range(2):  # twice: the staging buffer is reused
        cc.update_field(upd, F2)
    for plane in (CC_PLANE_ZHAT, CC_PLANE_SORTED, CC_PLANE_RANK2):
        assert np.array_equal(cc.get_plane(upd, plane, pts, n), cc.get_plane(ref, plane, pts, n))
    assert np.array_equal(cc.get_plane(upd, CC_PLANE_BINS, pts, n, bins=16),
                          cc.get_plane(ref, CC_PLANE_BINS, pts, n, bins=16))
    cc.free_field(upd)
    cc.free_field(ref)


@pytest.mark.parametrize("offset,scale", [(0.0, 1.0), (1e4, 1e-2), (-3e5, 7.0), (1e-30, 1e-33)])
def test_zhat_standardisation_accuracy(cc, offset, scale):
    """The unit-norm centred member vectors are within a few fp32 roundings of
    (v - mean) / sqrt(sum (v - mean)^2) evaluated in FP64, also when the mean
    is large against the spread (cancellation in the centring)."""
    rng = np.random.default_rng(11)
    for n in (32, 100, 1000):
        F = (offset + scale * rng.standard_normal((n, 2, 3, 4))).astype(np.float32)
        fid = cc.load_field(F)
        pts = np.arange(24, dtype=np.uint32)
        z = cc.get_plane(fid, 3, pts, n).astype(np.float64)
        V = F.reshape(n, -1).T.astype(np.float64)
        d = V - V.mean(axis=1, keepdims=True)
        ref = d / np.sqrt((d * d).sum(axis=1, keepdims=True))
        assert np.abs(z - ref).max() < 4 * 2.0 ** -24 * np.abs(ref).max(), (n, offset)
        cc.free_field(fid)


# ---------------------------------------------------------------- small config, all pairs
@pytest.mark.parametrize("kind,kw", [(oracle.PEARSON, {}), (oracle.SPEARMAN, {}),
                                     (oracle.MI_BINNED, {"bins": 8}), (oracle.MI_KSG, {"k": 3})],
                         ids=["pearson", "spearman", "hist8", "ksg3"])
def test_small_all_pairs_measures(cc, small, orc, kind, kw):
    from paper_2309_03308_gb300 import Params
    F, fid = small
    pa, pb = all_unique_pairs(F[0].size)
    assert pa.shape[0] == 523776
    got = cc.eval_pairs(fid, fid, Params(kind, **kw), pa, pb)
    ref = orc.eval_pairs(F, kind, pa, pb, **kw)
    err = np.abs(got.astype(np.float64) - ref)
    assert err.max() < TOL, (err.max(), int(err.argmax()))


def test_small_ksg_counts_bit_exact(cc, small, orc):
    F, fid = small
    rng = np.random.default_rng(4)
    P = F[0].size
    pa = rng.integers(0, P, 3000).astype(np.uint32)
    pb = rng.integers(0, P, 3000).astype(np.uint32)
    pb[:50] = pa[:50]  # identical points: x == y
    out, nx, ny, eps = cc.ksg_counts(fid, fid, 3, pa, pb, F.shape[0])
    ref, rnx, rny, reps = orc.eval_pairs(F, oracle.MI_KSG, pa, pb, k=3, want_ksg=True)
    assert np.array_equal(eps, reps)
    assert np.array_equal(nx, rnx) and np.array_equal(ny, rny)
    assert np.abs(out - ref).max() < TOL


# ---------------------------------------------------------------- focus config, sampled
def test_focus_measures_on_sampled_pairs(cc, focus, orc):
    from paper_2309_03308_gb300 import Params
    F, fid, ra, rb = focus
    c = configs.FOCUS
    pa, pb = cc.sample_pairs(ra, rb, c["sampler_seed"], 20000)
    for kind, kw in ((oracle.PEARSON, {}), (oracle.SPEARMAN, {}), (oracle.MI_BINNED, {"bins": 16}),
                     (oracle.MI_KSG, {"k": 10})):
        got = cc.eval_pairs(fid, fid, Params(kind, **kw), pa, pb)
        ref = orc.eval_pairs(F, kind, pa, pb, **kw)
        err = np.abs(got.astype(np.float64) - ref)
        assert err.max() < TOL, (kind, err.max())


def test_focus_ksg_counts_bit_exact(cc, focus, orc):
    F, fid, ra, rb = focus
    pa, pb = cc.sample_pairs(ra, rb, 11, 1500)
    out, nx, ny, eps = cc.ksg_counts(fid, fid, 10, pa, pb, F.shape[0])
    ref, rnx, rny, reps = orc.eval_pairs(F, oracle.MI_KSG, pa, pb, k=10, want_ksg=True)
    assert np.array_equal(eps, reps)
    assert np.array_equal(nx, rnx) and np.array_equal(ny, rny)


def test_ksg_n1000_counts_bit_exact(cc, orc):
    F = gen.field(2, 352, 256, 20, 1000, box=(64, 64, 0, 72, 70, 2))
    fid = cc.load_field(F)
    rng = np.random.default_rng(5)
    P = F[0].size
    pa = rng.integers(0, P, 120).astype(np.uint32)
    pb = rng.integers(0, P, 120).astype(np.uint32)
    out, nx, ny, eps = cc.ksg_counts(fid, fid, 10, pa, pb, 1000)
    ref, rnx, rny, reps = orc.eval_pairs(F, oracle.MI_KSG, pa, pb, k=10, want_ksg=True)
    assert np.array_equal(nx, rnx) and np.array_equal(ny, rny)
    assert np.abs(out - ref).max() < TOL
    from paper_2309_03308_gb300 import Params
    for kind in (oracle.PEARSON, oracle.SPEARMAN):
        got = cc.eval_pairs(fid, fid, Params(kind), pa, pb)
        assert np.abs(got - orc.eval_pairs(F, kind, pa, pb)).max() < TOL


@pytest.mark.parametrize("k", [1, 2, 5, 10, 16, 17, 31])
def test_ksg_k_range_and_ties(cc, orc, k):
    rng = np.random.default_rng(100 + k)
    F = rng.integers(0, 12, (32, 2, 3, 5)).astype(np.float32)  # many ties
    fid = cc.load_field(F)
    pa = rng.integers(0, 30, 400).astype(np.uint32)
    pb = rng.integers(0, 30, 400).astype(np.uint32)
    out, nx, ny, eps = cc.ksg_counts(fid, fid, k, pa, pb, 32)
    ref, rnx, rny, reps = orc.eval_pairs(F, oracle.MI_KSG, pa, pb, k=k, want_ksg=True)
    assert np.array_equal(eps, reps)
    assert np.array_equal(nx, rnx) and np.array_equal(ny, rny)
    assert np.abs(out - ref).max() < TOL


def test_ksg_paper_k_rule(cc, focus, orc):
    from paper_2309_03308_gb300 import Params
    F, fid, ra, rb = focus
    pa, pb = cc.sample_pairs(ra, rb, 12, 500)
    got = cc.eval_pairs(fid, fid, Params(oracle.MI_KSG, k=-1), pa, pb)
    ref = orc.eval_pairs(F, oracle.MI_KSG, pa, pb, k=orc.k_rule(100))
    assert np.abs(got - ref).max() < TOL


# ---------------------------------------------------------------- sampler
def test_sampler_matches_oracle(cc, focus, orc):
    F, fid, ra, rb = focus
    c = configs.FOCUS
    for (r1, r2, seed, stream, first) in ((ra, rb, 7, 0, 0), (ra, ra, 9, 3, 12345)):
        pa, pb = cc.sample_pairs(r1, r2, seed, 100000, stream=stream, first=first)
        A = oracle.box_points(c["X"], c["Y"], c["Z"], c["box_a"])
        B = A if r1 == r2 else oracle.box_points(c["X"], c["Y"], c["Z"], c["box_b"])
        ia, ib = orc.sample_pairs(seed, stream, first, len(A), len(B), r1 == r2, 100000)
        assert np.array_equal(pa, A[ia]) and np.array_equal(pb, B[ib])


# ---------------------------------------------------------------- segment extremes
def test_segment_extremes(cc, small, orc):
    from paper_2309_03308_gb300 import Params
    F, fid = small
    rng = np.random.default_rng(6)
    P = F[0].size
    sizes = [0, 1, 31, 32, 33, 500, 7]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    N = int(offs[-1])
    pa = rng.integers(0, P, N).astype(np.uint32)
    pb = rng.integers(0, P, N).astype(np.uint32)
    pb[10] = pb[11] = pa[10] = pa[11] = 3  # a tie on the max (r = 1)
    for kind, kw in ((oracle.PEARSON, {}), (oracle.MI_KSG, {"k": 3})):
        res = cc.segment_extremes(fid, Params(kind, **kw), pa, pb, offs)
        ref = orc.eval_pairs(F, kind, pa, pb, **kw)
        for s in range(len(sizes)):
            lo, hi = offs[s], offs[s + 1]
            assert res[s]["count"] == hi - lo
            if hi == lo:
                assert res[s]["max"] == -math.inf and res[s]["min"] == math.inf
                continue
            seg = ref[lo:hi]
            assert abs(res[s]["max"] - seg.max()) < TOL and abs(res[s]["min"] - seg.min()) < TOL
            assert lo <= res[s]["argmax"] < hi and abs(ref[res[s]["argmax"]] - seg.max()) < TOL
            assert lo <= res[s]["argmin"] < hi and abs(ref[res[s]["argmin"]] - seg.min()) < TOL


# ---------------------------------------------------------------- errors and edge cases
def test_errors(cc, small):
    from paper_2309_03308_gb300 import CCError, Params
    F, fid = small
    bad = F.copy()
    bad[3, 1, 2, 3] = np.nan
    with pytest.raises(CCError) as e:
        cc.load_field(bad)
    assert e.value.status == -4
    pa = np.array([0, 1 << 20], np.uint32)
    with pytest.raises(CCError) as e:
        cc.eval_pairs(fid, fid, Params(0), pa, pa)
    assert e.value.status == -1
    with pytest.raises(CCError):
        cc.eval_pairs(fid, fid, Params(oracle.MI_KSG, k=32), pa[:1], pa[:1])  # k > n-1
    with pytest.raises(CCError):
        cc.eval_pairs(fid, fid, Params(oracle.MI_BINNED, bins=17), pa[:1], pa[:1])
    empty = np.empty(0, np.uint32)
    assert cc.eval_pairs(fid, fid, Params(0), empty, empty).shape == (0,)
    # the context stays usable after errors
    ok = cc.eval_pairs(fid, fid, Params(0), pa[:1], pa[:1])
    assert abs(ok[0] - 1.0) < TOL


def test_device_buffers_and_torch_stream(small, orc):
    import torch
    from paper_2309_03308_gb300 import Context, Params
    F, _ = small
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = Context(0, stream=s.cuda_stream)
        fid = ctx.load_field(torch.from_numpy(F).cuda())
        pa, pb = all_unique_pairs(F[0].size)
        tpa = torch.from_numpy(pa.astype(np.int32)).cuda()
        tpb = torch.from_numpy(pb.astype(np.int32)).cuda()
        out = torch.empty(pa.shape[0], device="cuda")
        ctx.eval_pairs(fid, fid, Params(oracle.MI_KSG, k=3), tpa, tpb, out=out)
        ctx.sync()
        got = out.cpu().numpy()
        ctx.close()
    ref = orc.eval_pairs(F, oracle.MI_KSG, pa[:20000], pb[:20000], k=3)
    assert np.abs(got[:20000] - ref).max() < TOL


@pytest.mark.parametrize("mode", ["mean", "max"])
def test_aggregate_field(cc, orc, mode):
    """Block means / maxima of a field (Section 3.3) against the aggregate
    oracle, ragged boundary blocks included; the new field's planes and
    measures follow."""
    from oracle import agg
    from paper_2309_03308_gb300 import CC_AGG_MAX, CC_AGG_MEAN, CC_PEARSON, Params
    X, Y, Z, n = 37, 23, 9, 48
    F = gen.field(8, X, Y, Z, n)
    fid = cc.load_field(F)
    gid = cc.aggregate_field(fid, 4, 3, 2, CC_AGG_MEAN if mode == "mean" else CC_AGG_MAX)
    G = agg.aggregate(F, 4, 3, 2, mode)
    Pc = G[0].size
    pts = np.arange(Pc, dtype=np.uint32)
    got = cc.get_plane(gid, 2, pts, n)
    ref = np.sort(G.reshape(n, -1).T, axis=1)
    if mode == "max":
        assert np.array_equal(got, ref)
    else:
        ulp = np.spacing(np.abs(ref).astype(np.float32))
        assert np.all(np.abs(got - ref) <= ulp)
    pa, pb = all_unique_pairs(Pc)
    pa, pb = pa[::13].copy(), pb[::13].copy()
    vals = cc.eval_pairs(gid, gid, Params(CC_PEARSON), pa, pb)
    assert np.abs(vals - orc.eval_pairs(G, oracle.PEARSON, pa, pb)).max() < TOL
    cc.free_field(gid)
    cc.free_field(fid)
