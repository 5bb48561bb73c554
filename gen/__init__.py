"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws inputs only: ensemble fields (``field.c``), the cluster
fixture, and the workload geometry (``configs``). It contains none of the
correlation method's arithmetic, so both the FP64 oracle and the CUDA library
can consume what it produces without sharing code with each other.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgen.so")
_SRC = os.path.join(_HERE, "field.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile field.c into _build/libgen.so with gcc + OpenMP (host code only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.gen_field_box.restype = ctypes.c_int
            lib.gen_field_box.argtypes = [ctypes.c_uint64] + [ctypes.c_int] * 10 + [ctypes.c_void_p]
            lib.gen_clusters.restype = ctypes.c_int
            lib.gen_clusters.argtypes = [ctypes.c_uint64] + [ctypes.c_int] * 4 + [
                ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
            _lib = lib
    return _lib


def field(seed: int, X: int, Y: int, Z: int, n: int, box=None) -> np.ndarray:
    """Ensemble field of size X x Y x Z with n members, fp32, layout [n][Z][Y][X].

    ``box = (x0, y0, z0, x1, y1, z1)`` (half-open) returns only that sub-box,
    identical to the same voxels of the full field.
    """
    if box is None:
        box = (0, 0, 0, X, Y, Z)
    x0, y0, z0, x1, y1, z1 = box
    out = np.empty((n, z1 - z0, y1 - y0, x1 - x0), dtype=np.float32)
    rc = _load().gen_field_box(seed, X, Y, Z, n, x0, y0, z0, x1 - x0, y1 - y0, z1 - z0,
                               out.ctypes.data)
    if rc != 0:
        raise ValueError(f"gen_field_box failed ({rc})")
    return out


def coupled_field(F: np.ndarray, seed: int, shift: tuple[int, int], w_shift: float = 0.6,
                  w_noise: float = 0.8) -> np.ndarray:
    """A second variable on the grid of F ([n][Z][Y][X]): w_shift times F moved
    by shift = (dx, dy) voxels (periodic) plus w_noise times an independent
    field of the given seed. Stands in for a pair of physical variables (wind
    components) whose dependence is offset in space."""
    n, Z, Y, X = F.shape
    G = field(seed, X, Y, Z, n)
    return (w_shift * np.roll(F, shift=(shift[1], shift[0]), axis=(2, 3)) +
            w_noise * G).astype(np.float32)


def clusters(seed: int, X: int, Y: int, Z: int, n: int, centres) -> np.ndarray:
    """Cluster fixture (l-infinity decaying blend of one shared sequence and noise).

    ``centres`` is a list of (cx, cy, cz, radius). Voxels at a centre hold the
    same member vector, so their pairwise correlation is exactly 1.
    """
    c = np.ascontiguousarray(np.asarray(centres, dtype=np.int32).reshape(-1, 4))
    out = np.empty((n, Z, Y, X), dtype=np.float32)
    rc = _load().gen_clusters(seed, X, Y, Z, n, c.ctypes.data, c.shape[0], out.ctypes.data)
    if rc != 0:
        raise ValueError(f"gen_clusters failed ({rc})")
    return out


def gaussian_pair(seed: int, rho: float, n: int, reps: int) -> tuple[np.ndarray, np.ndarray]:
    """reps independent draws of n bivariate standard normals with correlation rho (fp64)."""
    rng = np.random.Generator(np.random.Philox(seed))
    a = rng.standard_normal((reps, n))
    b = rng.standard_normal((reps, n))
    return a, rho * a + np.sqrt(1.0 - rho * rho) * b
