"""KSG pair batches at 32 <= n <= 256, where a warp walks the samples of its
pairs as one stream and stages each pair into one of two slots: batches
smaller than a warp's lanes, batches long enough that every warp reuses its
slots many times, tie-heavy members, several k, and an out-of-range point id
in the middle of a batch. eps and both neighbour counts bit-exact
against the FP64 oracle, MI within 1e-5."""
import numpy as np
import pytest

import gen
import oracle

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


def check_counts(cc, orc, F, fid, k, pa, pb):
    n = F.shape[0]
    out, nx, ny, eps = cc.ksg_counts(fid, fid, k, pa, pb, n)
    ref, rnx, rny, reps = orc.eval_pairs(F, oracle.MI_KSG, pa, pb, k=k, want_ksg=True)
    assert np.array_equal(eps, reps)
    assert np.array_equal(nx, rnx) and np.array_equal(ny, rny)
    assert np.abs(out.astype(np.float64) - ref).max() < TOL


@pytest.mark.parametrize("npairs", [1, 2, 3, 5, 31, 33, 1000])
def test_small_batches(cc, orc, npairs):
    F = gen.field(41, 10, 8, 2, 100)
    fid = cc.load_field(F)
    rng = np.random.default_rng(npairs)
    P = F[0].size
    pa = rng.integers(0, P, npairs).astype(np.uint32)
    pb = rng.integers(0, P, npairs).astype(np.uint32)
    check_counts(cc, orc, F, fid, 10, pa, pb)
    cc.free_field(fid)


def test_long_batch_reuses_the_slots(cc, orc):
    # several pairs per warp, so each warp stages into and reuses both slots
    F = gen.field(43, 12, 10, 2, 100)
    fid = cc.load_field(F)
    rng = np.random.default_rng(3)
    P = F[0].size
    N = 60000
    pa = rng.integers(0, P, N).astype(np.uint32)
    pb = rng.integers(0, P, N).astype(np.uint32)
    pb[::97] = pa[::97]  # identical points: x == y
    check_counts(cc, orc, F, fid, 10, pa, pb)
    cc.free_field(fid)


@pytest.mark.parametrize("n,k", [(64, 1), (100, 10), (100, 31), (200, 4), (256, 16)])
def test_tie_heavy_members(cc, orc, n, k):
    rng = np.random.default_rng(n * 100 + k)
    F = rng.integers(0, 9, (n, 4, 3, 5)).astype(np.float32)
    fid = cc.load_field(F)
    P = F[0].size
    pa = rng.integers(0, P, 3000).astype(np.uint32)
    pb = rng.integers(0, P, 3000).astype(np.uint32)
    check_counts(cc, orc, F, fid, k, pa, pb)
    cc.free_field(fid)


def test_out_of_range_point_is_reported(cc, orc):
    from paper_2309_03308_gb300 import CCError, Params
    F = gen.field(47, 8, 8, 2, 100)
    fid = cc.load_field(F)
    P = F[0].size
    rng = np.random.default_rng(9)
    pa = rng.integers(0, P, 500).astype(np.uint32)
    pb = rng.integers(0, P, 500).astype(np.uint32)
    bad = pa.copy()
    bad[250] = P + 3
    with pytest.raises(CCError):
        cc.eval_pairs(fid, fid, Params(oracle.MI_KSG, k=10), bad, pb)
    # the context stays usable and exact afterwards
    check_counts(cc, orc, F, fid, 10, pa, pb)
    cc.free_field(fid)
