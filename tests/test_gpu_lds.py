"""Quasi-random pair samplers on the GPU (cc_sample_pairs_lds) against the
oracle's definitions (oracle/lds.py): bit-exact point pairs for Halton and
R6, cross and self region pairs, ragged boxes, offsets into the sequence."""
import numpy as np
import pytest

import gen
import oracle
from oracle import lds

pytestmark = pytest.mark.gpu
X, Y, Z = 37, 23, 9


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


@pytest.mark.parametrize("kind", ["halton", "r6"])
def test_lds_pairs_bit_exact(cc, kind):
    import torch
    from paper_2309_03308_gb300 import CC_LDS_HALTON, CC_LDS_R6
    code = {"halton": CC_LDS_HALTON, "r6": CC_LDS_R6}[kind]
    fid = cc.load_field(gen.field(3, X, Y, Z, 32))
    boxes = [(0, 0, 0, 13, 7, 3), (20, 5, 2, 37, 23, 9), (4, 11, 0, 5, 12, 9)]
    rids = cc.define_regions(fid, boxes)
    for (i, j, first, n) in [(0, 1, 0, 4000), (1, 0, 123456, 3000), (0, 0, 7, 3000),
                             (2, 2, 0, 500), (1, 2, (1 << 39) - 5000, 4000)]:
        pa, pb = cc.sample_pairs_lds(rids[i], rids[j], code, n, first=first)
        a, b = lds.sample_pairs_lds(kind, boxes[i], boxes[j], i == j, first, n)
        A = oracle.box_points(X, Y, Z, boxes[i])
        B = oracle.box_points(X, Y, Z, boxes[j])
        assert np.array_equal(pa, A[a]), (kind, i, j)
        assert np.array_equal(pb, B[b]), (kind, i, j)
    # device output, same values
    da = torch.empty(1000, dtype=torch.int32, device="cuda")
    db = torch.empty(1000, dtype=torch.int32, device="cuda")
    cc.sample_pairs_lds(rids[0], rids[1], code, 1000, first=11, pa=da, pb=db)
    ha, hb = cc.sample_pairs_lds(rids[0], rids[1], code, 1000, first=11)
    assert np.array_equal(da.cpu().numpy().view(np.uint32), ha)
    assert np.array_equal(db.cpu().numpy().view(np.uint32), hb)
    cc.free_field(fid)


def test_lds_argument_errors(cc):
    from paper_2309_03308_gb300 import CC_LDS_HALTON, CCError
    fid = cc.load_field(gen.field(3, X, Y, Z, 32))
    (r,) = cc.define_regions(fid, [(0, 0, 0, 4, 4, 2)])
    with pytest.raises(CCError):
        cc.sample_pairs_lds(r, r, 7, 10)
    with pytest.raises(CCError):
        cc.sample_pairs_lds(r, r, CC_LDS_HALTON, 10, first=1 << 40)
    cc.free_field(fid)
