"""FP64 CPU oracle (test infrastructure).

This package is the plain, slow, obviously correct reference for every
measure the CUDA library computes (arxiv 2309.03308, Section 3 and 3.2). It
shares no code with the library and the library never imports it. Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
load it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over pairs only);
this module marshals numpy arrays. ``mlp.py`` and ``gp.py`` hold the FP64
oracles of the learned surrogate and of the Gaussian-process sampler.

Parity pins (what fixes each function other than itself) are the tests in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

PEARSON, SPEARMAN, MI_BINNED, MI_KSG = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_libs: dict = {}

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_U64 = ctypes.c_uint64


def build(defines=(), force: bool = False) -> str:
    """Compile oracle.c with gcc (-O3, -ffp-contract=off, OpenMP).

    ``defines`` builds a variant (used by the tests that plant a mistake in
    the oracle to show a pin catches it); each variant gets its own file.
    """
    os.makedirs(_BUILD, exist_ok=True)
    tag = "_".join(d.replace("=", "-") for d in defines)
    so = os.path.join(_BUILD, f"liboracle{('_' + tag) if tag else ''}.so")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O3", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", *[f"-D{d}" for d in defines], _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, so)
    return so


class Oracle:
    """ctypes view of one build of oracle.c."""

    def __init__(self, defines=()):
        lib = ctypes.CDLL(build(defines))
        lib.or_eval_pairs.restype = _I
        lib.or_eval_pairs.argtypes = [_P, _I64, _P, _I64, _I, _I, _I, _I, _P, _P, _I64, _P, _P,
                                      _P, _P]
        lib.or_region_extremes.restype = _I
        lib.or_region_extremes.argtypes = [_P, _I64, _I, _P, _I64, _P, _I64, _I, _I, _I, _I, _P,
                                           _P]
        lib.or_rank2_points.argtypes = [_P, _I64, _I, _P, _I64, _P]
        lib.or_bins_points.argtypes = [_P, _I64, _I, _I, _P, _I64, _P]
        lib.or_digamma_int.restype = ctypes.c_double
        lib.or_digamma_int.argtypes = [_I]
        lib.or_k_rule.restype = _I
        lib.or_k_rule.argtypes = [_I]
        lib.or_philox4x64_10.argtypes = [_P, _P, _P]
        lib.or_sample_pairs.restype = _I
        lib.or_sample_pairs.argtypes = [_U64, _U64, _U64, _I64, _I64, _I, _I64, _P, _P]
        lib.or_threads.restype = _I
        lib.or_set_threads.argtypes = [_I]
        lib.or_pearson_vec.restype = ctypes.c_double
        lib.or_pearson_vec.argtypes = [_P, _P, _I]
        lib.or_hist_mi_bins.restype = ctypes.c_double
        lib.or_hist_mi_bins.argtypes = [_P, _P, _I, _I]
        lib.or_ksg_vec.restype = ctypes.c_double
        lib.or_ksg_vec.argtypes = [_P, _P, _I, _I, _P, _P, _P, _P]
        self.lib = lib

    # ------------------------------------------------------------------ helpers
    @staticmethod
    def _field(F):
        F = np.ascontiguousarray(F, dtype=np.float32)
        n = F.shape[0]
        return F.reshape(n, -1), n

    def threads(self) -> int:
        return self.lib.or_threads()

    def set_threads(self, t: int) -> None:
        self.lib.or_set_threads(int(t))

    # ------------------------------------------------------------------ measures
    def eval_pairs(self, F, kind, pa, pb, k=10, bins=16, Fb=None, want_ksg=False):
        """Measure between F[:, pa[t]] and Fb[:, pb[t]] (Fb defaults to F).

        F is [n][...] fp32. Returns values (fp64) or, with want_ksg, a tuple
        (values, nx, ny, eps) with the KSG counts and distances as [N][n].
        """
        F2, n = self._field(F)
        Fb2 = F2 if Fb is None else self._field(Fb)[0]
        pa = np.ascontiguousarray(pa, dtype=np.uint32)
        pb = np.ascontiguousarray(pb, dtype=np.uint32)
        N = pa.shape[0]
        out = np.empty(N, dtype=np.float64)
        nx = ny = eps = None
        if want_ksg:
            nx = np.empty((N, n), dtype=np.int32)
            ny = np.empty((N, n), dtype=np.int32)
            eps = np.empty((N, n), dtype=np.float32)
        rc = self.lib.or_eval_pairs(F2.ctypes.data, F2.shape[1], Fb2.ctypes.data, Fb2.shape[1], n,
                                    kind, k, bins, pa.ctypes.data, pb.ctypes.data, N,
                                    out.ctypes.data, nx.ctypes.data if want_ksg else None,
                                    ny.ctypes.data if want_ksg else None,
                                    eps.ctypes.data if want_ksg else None)
        if rc != 0:
            raise ValueError("or_eval_pairs: invalid arguments")
        return (out, nx, ny, eps) if want_ksg else out

    def pearson_vec(self, x, y) -> float:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        return self.lib.or_pearson_vec(x.ctypes.data, y.ctypes.data, x.shape[0])

    def ksg_vec(self, x, y, k):
        """KSG MI of two fp32 vectors; returns (mi, nx, ny, eps)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        n = x.shape[0]
        nx = np.empty(n, np.int32)
        ny = np.empty(n, np.int32)
        eps = np.empty(n, np.float32)
        work = np.empty(n, np.float32)
        mi = self.lib.or_ksg_vec(x.ctypes.data, y.ctypes.data, n, k, nx.ctypes.data,
                                 ny.ctypes.data, eps.ctypes.data, work.ctypes.data)
        return mi, nx, ny, eps

    def hist_mi_bins(self, bx, by, B) -> float:
        bx = np.ascontiguousarray(bx, dtype=np.uint8)
        by = np.ascontiguousarray(by, dtype=np.uint8)
        return self.lib.or_hist_mi_bins(bx.ctypes.data, by.ctypes.data, bx.shape[0], B)

    def rank2(self, F, pts) -> np.ndarray:
        """Doubled average ranks 2*rank (1-based) of the member vectors at pts: [len][n]."""
        F2, n = self._field(F)
        pts = np.ascontiguousarray(pts, dtype=np.uint32)
        out = np.empty((pts.shape[0], n), dtype=np.int32)
        self.lib.or_rank2_points(F2.ctypes.data, F2.shape[1], n, pts.ctypes.data, pts.shape[0],
                                 out.ctypes.data)
        return out

    def bins(self, F, pts, B) -> np.ndarray:
        """Equal-width bin ids of the member vectors at pts: [len][n] uint8."""
        F2, n = self._field(F)
        pts = np.ascontiguousarray(pts, dtype=np.uint32)
        out = np.empty((pts.shape[0], n), dtype=np.uint8)
        self.lib.or_bins_points(F2.ctypes.data, F2.shape[1], n, B, pts.ctypes.data, pts.shape[0],
                                out.ctypes.data)
        return out

    def digamma_int(self, m: int) -> float:
        return self.lib.or_digamma_int(int(m))

    def k_rule(self, n: int) -> int:
        return self.lib.or_k_rule(int(n))

    # ------------------------------------------------------------------ regions
    def region_extremes(self, F, A, B, self_pair, kind, k=10, bins=16, want_values=False):
        """Exhaustive extremes over a region pair. A, B are point-id arrays.

        Returns dict(max, min, argmax, argmin, count[, values]) with linear pair
        index a*len(B)+b (a < b only when self_pair).
        """
        F2, n = self._field(F)
        A = np.ascontiguousarray(A, dtype=np.uint32)
        B_ = np.ascontiguousarray(B, dtype=np.uint32)
        res = np.empty(5, dtype=np.float64)
        vals = np.full(A.shape[0] * B_.shape[0], np.nan) if want_values else None
        rc = self.lib.or_region_extremes(F2.ctypes.data, F2.shape[1], n, A.ctypes.data,
                                         A.shape[0], B_.ctypes.data, B_.shape[0], int(self_pair),
                                         kind, k, bins, res.ctypes.data,
                                         vals.ctypes.data if want_values else None)
        if rc != 0:
            raise ValueError("or_region_extremes failed")
        d = dict(max=res[0], min=res[1], argmax=int(res[2]), argmin=int(res[3]),
                 count=int(res[4]))
        if want_values:
            d["values"] = vals
        return d

    # ------------------------------------------------------------------ sampling
    def philox(self, ctr, key) -> np.ndarray:
        c = np.ascontiguousarray(ctr, dtype=np.uint64)
        k = np.ascontiguousarray(key, dtype=np.uint64)
        out = np.empty(4, dtype=np.uint64)
        self.lib.or_philox4x64_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
        return out

    def sample_pairs(self, seed, stream, first, na, nb, self_pair, N):
        ia = np.empty(N, dtype=np.uint32)
        ib = np.empty(N, dtype=np.uint32)
        rc = self.lib.or_sample_pairs(seed, stream, first, na, nb, int(self_pair), N,
                                      ia.ctypes.data, ib.ctypes.data)
        if rc != 0:
            raise ValueError("or_sample_pairs: invalid arguments")
        return ia, ib


def box_points(X, Y, Z, box) -> np.ndarray:
    """Linear point ids x + X*(y + Y*z) of a half-open box, x fastest."""
    x0, y0, z0, x1, y1, z1 = box
    z, y, x = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    return (x + X * (y + Y * z)).astype(np.uint32).ravel()


_default = None


def get() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle()
    return _default
