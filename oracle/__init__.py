"""Python access to the FP64 Lloyd k-means oracle (``kmref.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the library. It shares no code
with the GPU path; the only thing both sides take from the same place is the
seeded input generator (``synth``).

Every function here marshals numpy arrays into the C oracle and back; the
arithmetic is all in ``kmref.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmref.c")
_LIB = os.path.join(_HERE, "libkmref.so")
_lock = threading.Lock()
_lib = None


def compile_oracle(src: str, out: str) -> str:
    """gcc -O2 -fopenmp build of an oracle source file into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", src, "-o",
                           tmp, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_oracle(_SRC, _LIB)
    return _LIB


def bind(path: str):
    """Load an oracle shared library and declare its signatures."""
    lib = ctypes.CDLL(path)
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
    lib.kmref_set_threads.restype = ctypes.c_int
    lib.kmref_set_threads.argtypes = [ctypes.c_int]
    lib.kmref_assign.restype = ctypes.c_int
    lib.kmref_assign.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp, vp]
    lib.kmref_update.restype = ctypes.c_int
    lib.kmref_update.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp, vp]
    lib.kmref_objective.restype = dbl
    lib.kmref_objective.argtypes = [vp, i64, i32, vp, i32, vp]
    lib.kmref_step.restype = ctypes.c_int
    lib.kmref_step.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp, vp, vp]
    lib.kmref_run.restype = ctypes.c_int
    lib.kmref_run.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp, i32, dbl, vp, vp]
    lib.kmref_gda.restype = ctypes.c_int
    lib.kmref_gda.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp]
    lib.kmref_nb.restype = ctypes.c_int
    lib.kmref_nb.argtypes = [vp, i64, i32, vp, i32, vp, vp]
    lib.spaderef_densities.restype = ctypes.c_int
    lib.spaderef_densities.argtypes = [vp, i64, i32, dbl, dbl, i32, vp, vp, vp]
    lib.spaderef_count.restype = i64
    lib.spaderef_count.argtypes = [vp, i64, i32, i64, dbl]
    lib.spaderef_cover.restype = ctypes.c_int
    lib.spaderef_cover.argtypes = [vp, i64, i32, i64, dbl, vp, vp, vp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def _f32(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    return X


def _f64(C, d):
    C = np.ascontiguousarray(C, dtype=np.float64)
    return C.reshape(-1, d)


def _ptr(a):
    return a.ctypes.data if a is not None else None


class Oracle:
    """Thin marshalling layer over one loaded oracle library (the real one or a test mutant)."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else _load()

    def set_threads(self, n: int = 0) -> int:
        return int(self.lib.kmref_set_threads(n))

    def assign(self, X, C):
        """(assign int32[n], dmin f64[n], gap f64[n], second int32[n])."""
        X = _f32(X)
        n, d = X.shape
        C = _f64(C, d)
        k = C.shape[0]
        a = np.empty(n, np.int32)
        dmin = np.empty(n, np.float64)
        gap = np.empty(n, np.float64)
        second = np.empty(n, np.int32)
        rc = self.lib.kmref_assign(_ptr(X), n, d, _ptr(C), k, _ptr(a), _ptr(dmin), _ptr(gap),
                                   _ptr(second))
        if rc:
            raise ValueError(f"kmref_assign failed ({rc})")
        return a, dmin, gap, second

    def update(self, X, assign, Cprev):
        """(sums f64[k,d], counts int64[k], Cnew f64[k,d]) from a given assignment."""
        X = _f32(X)
        n, d = X.shape
        Cprev = _f64(Cprev, d)
        k = Cprev.shape[0]
        a = np.ascontiguousarray(assign, dtype=np.int32)
        sums = np.empty((k, d), np.float64)
        counts = np.empty(k, np.int64)
        Cnew = np.empty((k, d), np.float64)
        rc = self.lib.kmref_update(_ptr(X), n, d, _ptr(a), k, _ptr(Cprev), _ptr(sums),
                                   _ptr(counts), _ptr(Cnew))
        if rc:
            raise ValueError(f"kmref_update failed ({rc})")
        return sums, counts, Cnew

    def objective(self, X, C, assign) -> float:
        X = _f32(X)
        n, d = X.shape
        C = _f64(C, d)
        a = np.ascontiguousarray(assign, dtype=np.int32)
        return float(self.lib.kmref_objective(_ptr(X), n, d, _ptr(C), C.shape[0], _ptr(a)))

    def step(self, X, C):
        """One Lloyd step: dict(assign, sums, counts, C (new), objective, shift)."""
        X = _f32(X)
        n, d = X.shape
        C = _f64(C, d).copy()
        k = C.shape[0]
        a = np.empty(n, np.int32)
        sums = np.empty((k, d), np.float64)
        counts = np.empty(k, np.int64)
        J = ctypes.c_double()
        sh = ctypes.c_double()
        rc = self.lib.kmref_step(_ptr(X), n, d, _ptr(C), k, _ptr(a), _ptr(sums), _ptr(counts),
                                 ctypes.byref(J), ctypes.byref(sh))
        if rc:
            raise ValueError(f"kmref_step failed ({rc})")
        return dict(assign=a, sums=sums, counts=counts, C=C, objective=J.value, shift=sh.value)

    def run(self, X, C, iters: int, tol: float = 0.0):
        """Up to ``iters`` steps: dict(assign, sums, counts, C, objectives, iters_done)."""
        X = _f32(X)
        n, d = X.shape
        C = _f64(C, d).copy()
        k = C.shape[0]
        a = np.empty(n, np.int32)
        sums = np.empty((k, d), np.float64)
        counts = np.empty(k, np.int64)
        hist = np.zeros(max(iters, 1), np.float64)
        done = ctypes.c_int32()
        rc = self.lib.kmref_run(_ptr(X), n, d, _ptr(C), k, _ptr(a), _ptr(sums), _ptr(counts),
                                iters, tol, _ptr(hist), ctypes.byref(done))
        if rc:
            raise ValueError(f"kmref_run failed ({rc})")
        return dict(assign=a, sums=sums, counts=counts, C=C, objectives=hist[: done.value],
                    iters_done=done.value)


    # ---------------------------------------------------------------- keyed-reduce training

    def gda(self, X, y, ncls: int):
        """(phi f64[ncls], mu f64[ncls,d], sigma f64[d,d]): shared-covariance GDA."""
        X = _f32(X)
        n, d = X.shape
        yy = np.ascontiguousarray(y, dtype=np.int32)
        phi = np.empty(ncls, np.float64)
        mu = np.empty((ncls, d), np.float64)
        sigma = np.empty((d, d), np.float64)
        rc = self.lib.kmref_gda(_ptr(X), n, d, _ptr(yy), ncls, _ptr(phi), _ptr(mu), _ptr(sigma))
        if rc:
            raise ValueError(f"kmref_gda failed ({rc})")
        return phi, mu, sigma

    def nb(self, X, y, ncls: int):
        """(prior f64[ncls], theta f64[ncls,d]): multinomial naive Bayes, add-one smoothing."""
        X = _f32(X)
        n, d = X.shape
        yy = np.ascontiguousarray(y, dtype=np.int32)
        prior = np.empty(ncls, np.float64)
        theta = np.empty((ncls, d), np.float64)
        rc = self.lib.kmref_nb(_ptr(X), n, d, _ptr(yy), ncls, _ptr(prior), _ptr(theta))
        if rc:
            raise ValueError(f"kmref_nb failed ({rc})")
        return prior, theta


    # ---------------------------------------------------------------- SPADE downsampling

    def spade(self, X, apprx: float, kernel: float, policy: int = 0):
        """(densities int32[n], counts int32[n] (-1 for skipped rows), processed uint8[n]):
        the downsampling loop of Sec. 4.1 run sequentially (policy 0: generated code, 1: C++ snippet)."""
        X = _f32(X)
        n, d = X.shape
        dens = np.empty(n, np.int32)
        counts = np.empty(n, np.int32)
        proc = np.empty(n, np.uint8)
        rc = self.lib.spaderef_densities(_ptr(X), n, d, float(apprx), float(kernel), int(policy), _ptr(dens),
                                         _ptr(counts), _ptr(proc))
        if rc:
            raise ValueError(f"spaderef_densities failed ({rc})")
        return dens, counts, proc

    def spade_count(self, X, i: int, width: float) -> int:
        """#{j : D(i, j) < width} with the FP64 L1 distance."""
        X = _f32(X)
        n, d = X.shape
        c = int(self.lib.spaderef_count(_ptr(X), n, d, int(i), float(width)))
        if c < 0:
            raise ValueError("spaderef_count failed")
        return c

    def spade_cover(self, X, i: int, apprx: float, processed):
        """(first, last): lowest and highest processed row within apprx of row i (-1: none)."""
        X = _f32(X)
        n, d = X.shape
        p = np.ascontiguousarray(processed, dtype=np.uint8)
        first, last = ctypes.c_int64(), ctypes.c_int64()
        rc = self.lib.spaderef_cover(_ptr(X), n, d, int(i), float(apprx), _ptr(p), ctypes.byref(first),
                                     ctypes.byref(last))
        if rc:
            raise ValueError("spaderef_cover failed")
        return first.value, last.value


_default = None


def oracle() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default

