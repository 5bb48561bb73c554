"""The allocation-free all-pairs entry point (cc_all_pairs_static).

Callers that may not allocate device memory while they run (an interactive
per-frame loop, or a host application that keeps all device memory in its own
pool) get the same region-pair extremes as cc_all_pairs from planes they pass
in, with the scratch held in a static device array. The test compares it with
cc_all_pairs through the C ABI and with the FP64 oracle's exhaustive extremes,
on two calls in a row, for a cross and a self region pair. This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03308_gb300 import Context, _lib, build
    build.build()
    ctx = Context(0)
    yield torch, ctx, _lib.load()
    ctx.close()


def planes(torch, F, pts):
    """Member-major unit-norm centred planes [nk][lda] (FP64 standardisation, fp32 out)."""
    n = F.shape[0]
    x = torch.from_numpy(F.reshape(n, -1)[:, pts].astype(np.float64))
    x = x - x.mean(dim=0, keepdim=True)
    x = x / torch.sqrt((x * x).sum(dim=0, keepdim=True))
    nk = (n + 7) // 8 * 8
    lda = (len(pts) + 127) // 128 * 128
    out = torch.zeros((nk, lda), dtype=torch.float32)
    out[:n, :len(pts)] = x.to(torch.float32)
    return out.cuda(), nk, lda


def call_static(lib, za, lda, zb, ldb, nk, na, nb, self_pair, out):
    from paper_2309_03308_gb300 import _lib
    return lib.cc_all_pairs_static(za.data_ptr(), lda, zb.data_ptr(), ldb, nk, na, nb,
                                   int(self_pair), None, 0,
                                   ctypes.cast(out.data_ptr(), ctypes.POINTER(_lib.cc_rp_result)),
                                   None)


def as_result(buf):
    raw = buf.cpu().numpy().tobytes()
    mx, mn = np.frombuffer(raw[:8], np.float32)
    amax, amin, cnt = np.frombuffer(raw[8:32], np.uint64)
    return dict(max=float(mx), min=float(mn), argmax=int(amax), argmin=int(amin), count=int(cnt))


def test_static_matches_all_pairs_twice(env):
    torch, ctx, lib = env
    from paper_2309_03308_gb300 import Params
    X, Y, Z, n = 40, 24, 6, 50
    F = gen.field(17, X, Y, Z, n)
    fid = ctx.load_field(F)
    boxes = [(0, 0, 0, 17, 11, 6), (20, 5, 1, 40, 24, 5)]  # 1122 and 1520 points
    ra, rb = ctx.define_regions(fid, boxes)
    A = oracle.box_points(X, Y, Z, boxes[0])
    B = oracle.box_points(X, Y, Z, boxes[1])
    za, nk, lda = planes(torch, F, A)
    zb, _, ldb = planes(torch, F, B)
    out = torch.zeros(32, dtype=torch.uint8, device="cuda")
    orc = oracle.get()
    for (r1, r2, z1, l1, z2, l2, P1, P2) in ((ra, rb, za, lda, zb, ldb, A, B),
                                             (ra, ra, za, lda, za, lda, A, A)):
        ref = ctx.all_pairs(r1, r2, Params(0))
        exact = orc.region_extremes(F, P1, P2, r1 == r2, oracle.PEARSON)
        for _ in range(2):  # the static scratch keeps the previous call's contents
            out.fill_(0xFF)
            assert call_static(lib, z1, l1, z2, l2, nk, len(P1), len(P2), r1 == r2, out) == 0
            torch.cuda.synchronize()
            got = as_result(out)
            # the same result as the allocating entry point ...
            assert got["count"] == ref["count"]
            assert abs(got["max"] - ref["max"]) < TOL and abs(got["min"] - ref["min"]) < TOL
            # ... and as the FP64 oracle's exhaustive extremes
            assert got["count"] == exact["count"]
            assert abs(got["max"] - exact["max"]) < TOL and abs(got["min"] - exact["min"]) < TOL
            # the reported maximiser and minimiser are valid for the exact measure
            a, b = divmod(got["argmax"], len(P2))
            a2, b2 = divmod(got["argmin"], len(P2))
            v = oracle.get().eval_pairs(F, oracle.PEARSON, np.array([P1[a], P1[a2]]),
                                        np.array([P2[b], P2[b2]]))
            assert abs(v[0] - ref["max"]) < TOL and abs(v[1] - ref["min"]) < TOL


def test_static_rejects_oversized_request(env):
    torch, ctx, lib = env
    z = torch.zeros((8, 128), device="cuda")
    out = torch.zeros(32, dtype=torch.uint8, device="cuda")
    too_many = 128 * 257  # 257 x 257 tiles > 65,536
    from paper_2309_03308_gb300 import _lib
    rc = lib.cc_all_pairs_static(z.data_ptr(), too_many, z.data_ptr(), too_many, 8, too_many,
                                 too_many, 0, None, 0,
                                 ctypes.cast(out.data_ptr(), ctypes.POINTER(_lib.cc_rp_result)),
                                 None)
    assert rc == _lib.CC_ERR_INVALID_ARG
