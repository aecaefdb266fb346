"""Seeded synthetic Gaussian-mixture inputs for the Lloyd k-means workloads.

Holds no k-means arithmetic: it only draws points. Both the FP64 oracle's
tests and the GPU path's tests and benchmark take their inputs from here, so
the two sides see identical data without sharing any code of the method.

The generator itself is C (``synth.c``: SplitMix64 counters + Box-Muller),
compiled on first use with gcc into ``libkmsynth.so`` beside this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .workloads import SPADE_WORKLOADS, WORKLOADS, SpadeWorkload, Workload, batched_instances  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libkmsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libkmsynth.so`` (gcc, OpenMP) if missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, i32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            vp = ctypes.c_void_p
            lib.synth_splitmix64.restype = u64
            lib.synth_splitmix64.argtypes = [u64, u64]
            lib.synth_draw.restype = u64
            lib.synth_draw.argtypes = [u64, u64, u64]
            lib.synth_u01.restype = dbl
            lib.synth_u01.argtypes = [u64, u64, u64]
            lib.synth_normal.restype = dbl
            lib.synth_normal.argtypes = [u64, u64, u64]
            lib.synth_means.restype = None
            lib.synth_means.argtypes = [u64, i64, i64, dbl, vp]
            lib.synth_mixture_rows.restype = None
            lib.synth_mixture_rows.argtypes = [u64, i64, i64, i64, i64, vp, dbl, vp, vp]
            lib.synth_instance_shape.restype = None
            lib.synth_instance_shape.argtypes = [u64, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                                 ctypes.POINTER(i32)]
            _lib = lib
    return _lib


def splitmix64(state: int, i: int) -> int:
    return int(_load().synth_splitmix64(state, i))


def draw(seed: int, stream: int, ctr: int) -> int:
    return int(_load().synth_draw(seed, stream, ctr))


def u01(seed: int, stream: int, ctr: int) -> float:
    return float(_load().synth_u01(seed, stream, ctr))


def normal(seed: int, stream: int, e: int) -> float:
    return float(_load().synth_normal(seed, stream, e))


def means(seed: int, m: int, d: int, R: float) -> np.ndarray:
    mu = np.empty((m, d), dtype=np.float64)
    _load().synth_means(seed, m, d, R, mu.ctypes.data)
    return mu


def mixture(seed: int, n: int, d: int, m: int, R: float, sigma: float, *,
            row0: int = 0, out: np.ndarray | None = None, with_comp: bool = False):
    """Rows ``[row0, row0+n)`` of the seeded mixture as a C-contiguous float32 (n, d) array.

    ``out`` (optional) is a writable C-contiguous float32 array of that shape, e.g. the
    numpy view of a pinned host tensor. With ``with_comp`` the component index of every
    row is returned as well.
    """
    mu = means(seed, m, d, R)
    if out is None:
        out = np.empty((n, d), dtype=np.float32)
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.shape == (n, d)
    comp = np.empty(n, dtype=np.int32) if with_comp else None
    _load().synth_mixture_rows(seed, row0, n, d, m, mu.ctypes.data, sigma, out.ctypes.data,
                               comp.ctypes.data if comp is not None else None)
    return (out, comp) if with_comp else out


def multiscale_mixture(seed: int, n: int, d: int, m: int, R: float, sigma: float, span_log2: float):
    """The seeded mixture with component c (means and spread) scaled by 2^(-span_log2 c / (m - 1)),
    so that the component means' norms span a factor 2^span_log2; float32 (n, d)."""
    X, comp = mixture(seed, n, d, m, R, sigma, with_comp=True)
    f = np.exp2(-span_log2 * comp.astype(np.float64) / max(m - 1, 1)).astype(np.float32)
    return np.ascontiguousarray(X * f[:, None])


def instance_shape(seed: int):
    n, d, k = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _load().synth_instance_shape(seed, ctypes.byref(n), ctypes.byref(d), ctypes.byref(k))
    return int(n.value), int(d.value), int(k.value)


def workload_data(w: "Workload", *, rows: int | None = None, out: np.ndarray | None = None):
    """(X, C0) for a single-instance workload: X rows ``[0, rows)`` and C0 = the first k rows."""
    n = w.n if rows is None else rows
    X = mixture(w.seed, n, w.d, w.m, w.R, w.sigma, out=out)
    C0 = X[: w.k].copy() if n >= w.k else mixture(w.seed, w.k, w.d, w.m, w.R, w.sigma)
    return X, C0


def spade_data(w: "SpadeWorkload", *, rows: int | None = None) -> np.ndarray:
    """X rows ``[0, rows)`` of a SPADE downsampling workload."""
    return mixture(w.seed, w.n if rows is None else rows, w.d, w.m, w.R, w.sigma)
