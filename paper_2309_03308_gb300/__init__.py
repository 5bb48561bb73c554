"""GB300-native point-to-point correlation measures for 3D ensemble fields.

A thin Python view of the C ABI in ``include/ccorr.h`` (arxiv 2309.03308,
Section 3 and 3.2): every method marshals arguments and calls one entry point
of ``libccorr.so``; all arithmetic runs in the library's CUDA kernels.
PyTorch supplies device memory and streams. Arrays may be torch tensors (CUDA
or CPU) or numpy arrays; CPU arrays are passed as host memory.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (CC_AGG_MAX, CC_AGG_MEAN, CC_BF16, CC_FP8_E4M3, CC_FP32, CC_FP32_DOT2,
                   CC_LDS_HALTON, CC_LDS_R6,
                   CC_MI_BINNED, CC_MI_KSG, CC_PEARSON, CC_PLANE_BINS, CC_PLANE_RANK2,
                   CC_PLANE_SORTED, CC_PLANE_ZHAT, CC_SPEARMAN, CCError)

__all__ = ["Context", "Params", "CCError", "CC_PEARSON", "CC_SPEARMAN", "CC_MI_BINNED",
           "CC_MI_KSG", "CC_FP32", "CC_BF16", "CC_FP8_E4M3", "CC_FP32_DOT2", "CC_LDS_HALTON",
           "CC_LDS_R6", "CC_AGG_MEAN", "CC_AGG_MAX"]


@dataclass
class Params:
    """cc_params: measure, KSG k (-1 = paper rule ceil(3n/100)), bins, precision."""
    measure: int = CC_PEARSON
    k: int = 10
    bins: int = 16
    precision: int = CC_FP32

    def c(self) -> _lib.cc_params:
        return _lib.cc_params(self.measure, self.k, self.bins, self.precision, 0)


def _ptr(a):
    """(pointer, is_device) of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


class Context:
    """One cc_ctx: a device, a stream, loaded fields and regions."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        s = int(stream) if stream is not None else None
        self._check(self.lib.cc_create(device, s, ctypes.byref(h)), ctx=None)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.cc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, status, ctx="self"):
        if status != 0:
            msg = ""
            if ctx == "self" and self.h:
                m = self.lib.cc_last_error(self.h)
                msg = m.decode() if m else ""
            raise CCError(status, msg)

    # --------------------------------------------------------------- fields
    def cc_load_field(self, data, X: int, Y: int, Z: int, n: int) -> int:
        p, dev = _ptr(data)
        fid = ctypes.c_int32()
        self._check(self.lib.cc_load_field(self.h, p, dev, X, Y, Z, n, ctypes.byref(fid)))
        return fid.value

    def load_field(self, data) -> int:
        """Load an fp32 [n][Z][Y][X] array (torch or numpy)."""
        n, Z, Y, X = data.shape
        return self.cc_load_field(data, X, Y, Z, n)

    def update_field(self, fid: int, data):
        """Replace a loaded field's values (same shape) and recompute its planes in place."""
        p, dev = _ptr(data)
        self._check(self.lib.cc_update_field(self.h, fid, p, dev))

    def aggregate_field(self, fid: int, bx: int, by: int, bz: int, mode: int = 0) -> int:
        """New field of block means (mode CC_AGG_MEAN) or maxima (CC_AGG_MAX)."""
        out = ctypes.c_int32()
        self._check(self.lib.cc_aggregate_field(self.h, fid, bx, by, bz, mode, ctypes.byref(out)))
        return out.value

    def free_field(self, fid: int):
        self._check(self.lib.cc_free_field(self.h, fid))

    def get_plane(self, fid: int, plane: int, pts, n: int, bins: int = 0) -> np.ndarray:
        pts = np.ascontiguousarray(pts, dtype=np.uint32)
        dt = {CC_PLANE_RANK2: np.int32, CC_PLANE_BINS: np.uint8, CC_PLANE_SORTED: np.float32,
              CC_PLANE_ZHAT: np.float32}[plane]
        out = np.empty((pts.shape[0], n), dtype=dt)
        self._check(self.lib.cc_get_plane(self.h, fid, plane, bins, pts.ctypes.data,
                                          pts.shape[0], out.ctypes.data))
        return out

    # --------------------------------------------------------------- regions
    def define_regions(self, fid: int, boxes) -> list:
        arr = (_lib.cc_box * len(boxes))(*[_lib.cc_box(*b) for b in boxes])
        ids = (ctypes.c_int32 * len(boxes))()
        self._check(self.lib.cc_define_regions(self.h, fid, arr, len(boxes), ids))
        return list(ids)

    def partition_regular(self, fid: int, bx: int, by: int, bz: int, cap: int = 1 << 20) -> list:
        ids = (ctypes.c_int32 * cap)()
        cnt = ctypes.c_int()
        self._check(self.lib.cc_partition_regular(self.h, fid, bx, by, bz, ids, cap,
                                                  ctypes.byref(cnt)))
        return list(ids[:cnt.value])

    def region_info(self, rid: int):
        npts = ctypes.c_int64()
        box = _lib.cc_box()
        self._check(self.lib.cc_region_info(self.h, rid, ctypes.byref(npts), ctypes.byref(box)))
        return npts.value, (box.x0, box.y0, box.z0, box.x1, box.y1, box.z1)

    # --------------------------------------------------------------- sampling / evaluation
    def sample_pairs(self, ra: int, rb: int, seed: int, n_pairs: int, stream: int = 0,
                     first: int = 0, pa=None, pb=None):
        """Seeded uniform pairs; fills pa/pb (allocated as numpy when None)."""
        if pa is None:
            pa = np.empty(n_pairs, np.uint32)
            pb = np.empty(n_pairs, np.uint32)
        a, dev = _ptr(pa)
        b, _ = _ptr(pb)
        self._check(self.lib.cc_sample_pairs(self.h, ra, rb, seed, stream, first, n_pairs, a, b,
                                             dev))
        return pa, pb

    def sample_pairs_lds(self, ra: int, rb: int, kind: int, n_pairs: int, first: int = 0,
                         pa=None, pb=None):
        """Quasi-random pairs (kind CC_LDS_HALTON or CC_LDS_R6); numpy when pa is None."""
        if pa is None:
            pa = np.empty(n_pairs, np.uint32)
            pb = np.empty(n_pairs, np.uint32)
        a, dev = _ptr(pa)
        b, _ = _ptr(pb)
        self._check(self.lib.cc_sample_pairs_lds(self.h, ra, rb, kind, first, n_pairs, a, b, dev))
        return pa, pb

    def eval_pairs(self, fa: int, fb: int, params: Params, pa, pb, out=None):
        n_pairs = int(pa.shape[0])
        a, pdev = _ptr(pa)
        b, _ = _ptr(pb)
        if out is None:
            out = np.empty(n_pairs, np.float32)
        o, odev = _ptr(out)
        prm = params.c()
        self._check(self.lib.cc_eval_pairs(self.h, fa, fb, ctypes.byref(prm), a, b, n_pairs, pdev,
                                           o, odev))
        return out

    def ksg_counts(self, fa: int, fb: int, k: int, pa, pb, n: int):
        pa = np.ascontiguousarray(pa, np.uint32)
        pb = np.ascontiguousarray(pb, np.uint32)
        N = pa.shape[0]
        out = np.empty(N, np.float32)
        nx = np.empty((N, n), np.int32)
        ny = np.empty((N, n), np.int32)
        eps = np.empty((N, n), np.float32)
        self._check(self.lib.cc_ksg_counts(self.h, fa, fb, k, pa.ctypes.data, pb.ctypes.data, N,
                                           out.ctypes.data, nx.ctypes.data, ny.ctypes.data,
                                           eps.ctypes.data))
        return out, nx, ny, eps

    def segment_extremes(self, fid: int, params: Params, pa, pb, seg_offsets, values=None,
                         field_b: int | None = None):
        """Per-segment extremes of pairs (pa[t] of field fid, pb[t] of field_b,
        default fid)."""
        offs = np.ascontiguousarray(seg_offsets, np.int64)
        n_seg = offs.shape[0] - 1
        a, pdev = _ptr(pa)
        b, _ = _ptr(pb)
        v = _ptr(values)[0] if values is not None else None
        res = (_lib.cc_rp_result * max(n_seg, 1))()
        prm = params.c()
        fb = fid if field_b is None else field_b
        self._check(self.lib.cc_segment_extremes2(self.h, fid, fb, ctypes.byref(prm), a, b, pdev,
                                                  offs.ctypes.data, n_seg, v, res))
        return [_res(r) for r in res[:n_seg]]

    def all_pairs(self, ra: int, rb: int, params: Params, values=None, ld: int = 0):
        v = None
        if values is not None:
            v, dev = _ptr(values)
            if not dev:
                raise ValueError("values must be device memory")
            ld = ld or int(values.shape[-1])
        res = _lib.cc_rp_result()
        prm = params.c()
        self._check(self.lib.cc_all_pairs(self.h, ra, rb, ctypes.byref(prm), v, ld,
                                          ctypes.byref(res)))
        return _res(res)

    def all_pairs_topk(self, ra: int, rb: int, params: Params, topk: int = 0):
        """Reduced-precision all-pairs: (extremes, top ids, top values, certificate)."""
        ids = np.empty(max(topk, 1), np.uint64)
        vals = np.empty(max(topk, 1), np.float32)
        res = _lib.cc_rp_result()
        info = _lib.cc_mixed_info()
        prm = params.c()
        self._check(self.lib.cc_all_pairs_topk(self.h, ra, rb, ctypes.byref(prm), topk,
                                               ids.ctypes.data, vals.ctypes.data,
                                               ctypes.byref(res), ctypes.byref(info)))
        cert = {f: getattr(info, f) for f, _ in _lib.cc_mixed_info._fields_}
        return _res(res), ids[:topk], vals[:topk], cert

    def all_pairs_approx(self, ra: int, rb: int, params: Params):
        """Approximate per-(row, 32-column chunk) extremes of the reduced-precision
        contraction: (cmax [chunks][|A|], cmin [chunks][|A|], certified bound)."""
        na, _ = self.region_info(ra)
        nb, _ = self.region_info(rb)
        chunks = (nb + 31) // 32
        cmax = np.empty((chunks, na), np.float32)
        cmin = np.empty((chunks, na), np.float32)
        bound = ctypes.c_float()
        prm = params.c()
        self._check(self.lib.cc_all_pairs_approx(self.h, ra, rb, ctypes.byref(prm),
                                                 cmax.ctypes.data, cmin.ctypes.data,
                                                 ctypes.byref(bound)))
        return cmax, cmin, bound.value

    def bos_create(self, fid: int, rp_a, rp_b, pool=2048, per_round=32, rounds=30,
                   shortlist=128, kappa=0.5, objective=CC_MI_KSG, k=10, bins=16, seed=3,
                   field_b: int | None = None, local_picks=0, local_scale=0.0625):
        """Batched BOS state over region pairs (rp_a[i], rp_b[i]) of field fid;
        with field_b, the second point of each pair is read from that field
        (regions rp_b[i] belong to it): the inter-variable matrix. local_picks
        proposals per round (from the second) perturb the two best samples."""
        a = np.ascontiguousarray(rp_a, np.int32)
        b = np.ascontiguousarray(rp_b, np.int32)
        prm = _lib.cc_bos_params(pool, per_round, rounds, shortlist, kappa, objective, k, bins,
                                 seed, local_picks, local_scale)
        h = ctypes.c_void_p()
        fb = fid if field_b is None else field_b
        self._check(self.lib.cc_bos_create2(self.h, fid, fb, a.ctypes.data, b.ctypes.data,
                                            len(a), ctypes.byref(prm), ctypes.byref(h)))
        return Bos(self, h, len(a), prm)

    def sync(self):
        self._check(self.lib.cc_sync(self.h))


class Bos:
    """cc_bos handle: batched Bayesian optimal sampling over region pairs."""

    def __init__(self, ctx: Context, h, n_rp: int, prm):
        self.ctx, self.h, self.n_rp, self.prm = ctx, h, n_rp, prm

    def set_prior(self, prior):
        p, dev = _ptr(prior) if prior is not None else (None, 0)
        self.ctx._check(self.ctx.lib.cc_bos_set_prior(self.ctx.h, self.h, p, dev))

    def run(self, rounds: int, use_graph: bool = True):
        self.ctx._check(self.ctx.lib.cc_bos_run(self.ctx.h, self.h, rounds, int(use_graph)))

    def results(self):
        """[4][n_rp] dicts (Pearson, Spearman, binned MI, KSG); argmax = (a << 32) | b."""
        res = (_lib.cc_rp_result * (4 * self.n_rp))()
        self.ctx._check(self.ctx.lib.cc_bos_results(self.ctx.h, self.h, res))
        return [[_res(res[m * self.n_rp + i]) for i in range(self.n_rp)] for m in range(4)]

    def inspect(self, rp: int):
        Q, R, T = self.prm.pool, self.prm.per_round, self.prm.rounds
        pool = np.empty((Q, 6), np.float32)
        mu = np.empty(Q, np.float32)
        var = np.empty(Q, np.float32)
        obs = np.empty(R * T, np.int32)
        y = np.empty(R * T, np.float32)
        pa = np.empty(R, np.uint32)
        pb = np.empty(R, np.uint32)
        vals = np.empty((4, R), np.float32)
        n = ctypes.c_int32()
        self.ctx._check(self.ctx.lib.cc_bos_inspect(
            self.ctx.h, self.h, rp, pool.ctypes.data, mu.ctypes.data, var.ctypes.data,
            obs.ctypes.data, y.ctypes.data, pa.ctypes.data, pb.ctypes.data, vals.ctypes.data,
            ctypes.byref(n)))
        s = n.value
        return dict(pool=pool, mu=mu, var=var, obs=obs[:s], y=y[:s], pa=pa, pb=pb, vals=vals)

    def samples(self, rp: int):
        """Every evaluated sample of region pair rp in order: (theta [n][6], objective [n])."""
        R, T = self.prm.per_round, self.prm.rounds
        theta = np.empty((R * T, 6), np.float32)
        y = np.empty(R * T, np.float32)
        n = ctypes.c_int32()
        self.ctx._check(self.ctx.lib.cc_bos_samples(self.ctx.h, self.h, rp, theta.ctypes.data,
                                                    y.ctypes.data, ctypes.byref(n)))
        return theta[:n.value], y[:n.value]

    def close(self):
        if self.h:
            self.ctx.lib.cc_bos_destroy(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """cc_sur handle: the learned pairwise predictor (BF16 training/inference)."""

    def __init__(self, ctx: Context, n_members: int, seed: int = 0):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._check(ctx.lib.cc_sur_create(ctx.h, n_members, seed, ctypes.byref(h)))
        self.h = h

    def params(self):
        n = ctypes.c_int64()
        m, s = ctypes.c_float(), ctypes.c_float()
        self.ctx._check(self.ctx.lib.cc_sur_get_params(self.ctx.h, self.h, None, ctypes.byref(n),
                                                       ctypes.byref(m), ctypes.byref(s)))
        out = np.empty(n.value, np.float32)
        self.ctx._check(self.ctx.lib.cc_sur_get_params(self.ctx.h, self.h, out.ctypes.data, None,
                                                       None, None))
        return out, m.value, s.value

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        self.ctx._check(self.ctx.lib.cc_sur_set_params(self.ctx.h, self.h, flat.ctypes.data))

    def set_target_scale(self, mean: float, sd: float):
        self.ctx._check(self.ctx.lib.cc_sur_set_target_scale(self.ctx.h, self.h, mean, sd))

    def loss_grad(self, fid: int, pa, pb, target):
        pa = np.ascontiguousarray(pa, np.uint32)
        pb = np.ascontiguousarray(pb, np.uint32)
        t = np.ascontiguousarray(target, np.float32)
        grad = np.empty(self.params()[0].shape[0], np.float32)
        loss = ctypes.c_float()
        self.ctx._check(self.ctx.lib.cc_sur_loss_grad(self.ctx.h, self.h, fid, pa.ctypes.data,
                                                      pb.ctypes.data, t.ctypes.data, len(pa),
                                                      ctypes.byref(loss), grad.ctypes.data))
        return loss.value, grad

    def train(self, fid: int, pa, pb, target, epochs=1, batch=4096, lr=1e-3, seed=0):
        a, dev = _ptr(pa)
        b, _ = _ptr(pb)
        t, _ = _ptr(target)
        losses = np.empty(max(epochs, 1), np.float32)
        self.ctx._check(self.ctx.lib.cc_sur_train(self.ctx.h, self.h, fid, a, b, t,
                                                  int(pa.shape[0]), dev, epochs, batch, lr, seed,
                                                  losses.ctypes.data))
        return losses[:epochs]

    def predict(self, fid: int, pa, pb, out=None):
        a, pdev = _ptr(pa)
        b, _ = _ptr(pb)
        if out is None:
            out = np.empty(int(pa.shape[0]), np.float32)
        o, odev = _ptr(out)
        self.ctx._check(self.ctx.lib.cc_sur_predict(self.ctx.h, self.h, fid, a, b,
                                                    int(pa.shape[0]), pdev, o, odev))
        return out

    def screen(self, ra: int, rb: int, topk: int):
        ids = np.empty(topk, np.uint64)
        preds = np.empty(topk, np.float32)
        self.ctx._check(self.ctx.lib.cc_sur_screen(self.ctx.h, self.h, ra, rb, topk,
                                                   ids.ctypes.data, preds.ctypes.data))
        return ids, preds

    def screen_verify(self, ra: int, rb: int, budget: int, params: Params):
        """Exact extremes over the `budget` pairs the surrogate ranks highest."""
        res = _lib.cc_rp_result()
        prm = params.c()
        self.ctx._check(self.ctx.lib.cc_sur_screen_verify(self.ctx.h, self.h, ra, rb, budget,
                                                          ctypes.byref(prm), ctypes.byref(res)))
        return _res(res)

    def close(self):
        if self.h:
            self.ctx.lib.cc_sur_destroy(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by libccorr.so in this process so far."""
    c = ctypes.c_uint64()
    _lib.load().cc_launch_count(ctypes.byref(c))
    return c.value


def _res(r) -> dict:
    return dict(max=r.max, min=r.min, argmax=r.argmax, argmin=r.argmin, count=r.count)
