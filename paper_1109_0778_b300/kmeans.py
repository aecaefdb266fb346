"""Python binding of libkmeans.so (include/kmeans.h): argument marshalling only.

Every stage of the Lloyd step runs in the library's CUDA kernels; this module
checks tensor types and shapes, passes raw pointers and sizes through ctypes,
and turns a km_status into an exception. There is no CPU path: if the shared
library is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkmeans.so")

KM_OK, KM_EINVAL, KM_ECUDA, KM_ENOMEM, KM_EUNSUPPORTED, KM_ETIMEOUT, KM_ENONFINITE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "KM_OK", -1: "KM_EINVAL", -2: "KM_ECUDA", -3: "KM_ENOMEM", -4: "KM_EUNSUPPORTED",
                -5: "KM_ETIMEOUT", -6: "KM_ENONFINITE"}
PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2, "bf16x3": 3}
STAGES = ("xnorm", "prep", "assign", "recheck", "count", "scan", "scatter", "segsum", "divide")

#: Entry points declared in include/kmeans.h (checked by the ABI test).
EXPORTS = ("kmeans_default_opts", "kmeans_step", "kmeans_run", "kmeans_step_ex", "kmeans_run_ex",
           "kmeans_run_host", "kmeans_last_error", "kmeans_version", "kmeans_reduce_noalloc",
           "kmeans_run_batched", "kmeans_gda_train", "kmeans_nb_train", "kmeans_spade_densities",
           "kmeans_probe_mma", "kmeans_probe_ffma", "kmeans_step_partial", "kmeans_apply_partials")
SPADE_POLICY = {"last": 0, "first": 1}


class KMeansError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("recheck", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("reuse_x", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class Instance(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("k", ctypes.c_int32),
                ("C", ctypes.c_void_p), ("assign", ctypes.c_void_p), ("sums", ctypes.c_void_p),
                ("counts", ctypes.c_void_p)]


class SpadeStats(ctypes.Structure):
    _fields_ = [("n_evaluated", ctypes.c_int64), ("n_computed", ctypes.c_int64),
                ("n_found_pairs", ctypes.c_int64), ("n_exact", ctypes.c_int64),
                ("batches", ctypes.c_int32), ("overflow_batches", ctypes.c_int32),
                ("ms", ctypes.c_float), ("ms_pairs", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("objective", ctypes.c_double), ("shift", ctypes.c_double),
                ("n_changed", ctypes.c_int64), ("n_flagged", ctypes.c_int64),
                ("n_full", ctypes.c_int64), ("n_empty", ctypes.c_int32),
                ("iters_done", ctypes.c_int32), ("ms", ctypes.c_float),
                ("launches", ctypes.c_int32), ("stage_ms", ctypes.c_float * 12),
                ("n_queued", ctypes.c_int64), ("iters_bf16", ctypes.c_int32), ("batch_shape", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "stage_ms"}
        d["stage_ms"] = {name: float(self.stage_ms[i]) for i, name in enumerate(STAGES)}
        return d


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libkmeans.so not built at {path}: run paper_1109_0778_b300/build.py")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    P = ctypes.POINTER
    lib.kmeans_default_opts.restype = None
    lib.kmeans_default_opts.argtypes = [P(Opts)]
    lib.kmeans_step.restype = ctypes.c_int
    lib.kmeans_step.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp]
    lib.kmeans_run.restype = ctypes.c_int
    lib.kmeans_run.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp, i32, dbl]
    lib.kmeans_step_ex.restype = ctypes.c_int
    lib.kmeans_step_ex.argtypes = [P(Opts), vp, i64, i32, vp, i32, vp, vp, vp, P(Stats)]
    lib.kmeans_run_ex.restype = ctypes.c_int
    lib.kmeans_run_ex.argtypes = [P(Opts), vp, i64, i32, vp, i32, vp, vp, vp, i32, dbl, P(Stats)]
    lib.kmeans_run_host.restype = ctypes.c_int
    lib.kmeans_run_host.argtypes = [P(Opts), vp, i64, i32, vp, i32, vp, vp, vp, i32, dbl, P(Stats)]
    lib.kmeans_last_error.restype = ctypes.c_char_p
    lib.kmeans_last_error.argtypes = []
    lib.kmeans_version.restype = ctypes.c_int32
    lib.kmeans_version.argtypes = []
    lib.kmeans_run_batched.restype = ctypes.c_int
    lib.kmeans_run_batched.argtypes = [P(Opts), P(Instance), i32, i32, dbl, P(Stats)]
    lib.kmeans_reduce_noalloc.restype = ctypes.c_int
    lib.kmeans_reduce_noalloc.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp, P(dbl), vp]
    lib.kmeans_gda_train.restype = ctypes.c_int
    lib.kmeans_gda_train.argtypes = [P(Opts), vp, i64, i32, vp, i32, vp, vp, vp]
    lib.kmeans_nb_train.restype = ctypes.c_int
    lib.kmeans_nb_train.argtypes = [P(Opts), vp, i64, i32, vp, i32, vp, vp]
    lib.kmeans_spade_densities.restype = ctypes.c_int
    lib.kmeans_spade_densities.argtypes = [P(Opts), vp, i64, i32, dbl, dbl, i32, vp, vp, vp, P(SpadeStats)]
    lib.kmeans_step_partial.restype = ctypes.c_int
    lib.kmeans_step_partial.argtypes = [P(Opts), vp, i64, i32, vp, i32, vp, vp, P(Stats)]
    lib.kmeans_apply_partials.restype = ctypes.c_int
    lib.kmeans_apply_partials.argtypes = [P(Opts), vp, i32, i32, vp, vp, vp, P(Stats)]
    lib.kmeans_probe_mma.restype = ctypes.c_int
    lib.kmeans_probe_mma.argtypes = [i32, vp, vp, i32, vp, vp]
    lib.kmeans_probe_ffma.restype = ctypes.c_int
    lib.kmeans_probe_ffma.argtypes = [i32, i32, P(dbl), P(ctypes.c_float), vp]
    return lib


_lib = load()


def lib():
    return _lib


def _check(rc: int):
    if rc != KM_OK:
        raise KMeansError(rc, _lib.kmeans_last_error().decode())


def make_opts(precision: str = "fp32", recheck: bool = True, stream=None, profile: bool = False,
              warm_start: bool = False, deterministic: bool = False, reuse_x: bool = False) -> Opts:
    o = Opts()
    _lib.kmeans_default_opts(ctypes.byref(o))
    o.precision = PRECISION[precision]
    o.recheck = 1 if recheck else 0
    o.profile = 1 if profile else 0
    o.warm_start = 1 if warm_start else 0
    o.deterministic = 1 if deterministic else 0
    o.reuse_x = 1 if reuse_x else 0
    o.stream = stream
    return o


def _stream_handle(stream):
    import torch

    if stream is None:
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _check_tensors(X, C, assign, sums, counts):
    import torch

    n, d = X.shape
    k = C.shape[0]
    for name, t, dt, shape in (("X", X, torch.float32, (n, d)), ("C", C, torch.float32, (k, d)),
                               ("assign", assign, torch.int32, (n,)), ("sums", sums, torch.float32, (k, d)),
                               ("counts", counts, torch.int32, (k,))):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dt} tensor of shape {shape}")
    return n, d, k


@dataclass
class Outputs:
    assign: "object"
    sums: "object"
    counts: "object"
    stats: dict


def alloc_outputs(X, C):
    import torch

    n, _ = X.shape
    k, d = C.shape
    return (torch.empty(n, dtype=torch.int32, device=X.device),
            torch.empty(k, d, dtype=torch.float32, device=X.device),
            torch.empty(k, dtype=torch.int32, device=X.device))


def step(X, C, assign=None, sums=None, counts=None, *, precision="fp32", recheck=True, stream=None,
         profile=False, warm_start=False, deterministic=False, reuse_x=False) -> Outputs:
    """One Lloyd step on device tensors; C is updated in place (kmeans_step_ex)."""
    if assign is None:
        assign, sums, counts = alloc_outputs(X, C)
    n, d, k = _check_tensors(X, C, assign, sums, counts)
    o = make_opts(precision, recheck, _stream_handle(stream), profile, warm_start, deterministic, reuse_x)
    st = Stats()
    _check(_lib.kmeans_step_ex(ctypes.byref(o), X.data_ptr(), n, d, C.data_ptr(), k, assign.data_ptr(),
                               sums.data_ptr(), counts.data_ptr(), ctypes.byref(st)))
    return Outputs(assign, sums, counts, st.as_dict())


def run(X, C, iters, tol=0.0, assign=None, sums=None, counts=None, *, precision="fp32", recheck=True,
        stream=None, profile=False, warm_start=False, deterministic=False, reuse_x=False) -> Outputs:
    """Up to ``iters`` Lloyd steps on device tensors; C is updated in place (kmeans_run_ex)."""
    if assign is None:
        assign, sums, counts = alloc_outputs(X, C)
    n, d, k = _check_tensors(X, C, assign, sums, counts)
    o = make_opts(precision, recheck, _stream_handle(stream), profile, warm_start, deterministic, reuse_x)
    st = Stats()
    _check(_lib.kmeans_run_ex(ctypes.byref(o), X.data_ptr(), n, d, C.data_ptr(), k, assign.data_ptr(),
                              sums.data_ptr(), counts.data_ptr(), int(iters), float(tol), ctypes.byref(st)))
    return Outputs(assign, sums, counts, st.as_dict())


def run_host(X, C, iters, tol=0.0, assign=None, sums=None, counts=None, *, precision="fp32", recheck=True,
             stream=None):
    """kmeans_run_host on host arrays (numpy arrays or CPU tensors, pinned or not).

    C is updated in place; assign, sums and counts are filled. Returns the stats dict.
    """
    import numpy as np

    def ptr(a):
        return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()

    n, d = X.shape
    k = C.shape[0]
    o = make_opts(precision, recheck, stream)
    st = Stats()
    _check(_lib.kmeans_run_host(ctypes.byref(o), ptr(X), n, d, ptr(C), k, ptr(assign), ptr(sums), ptr(counts),
                                int(iters), float(tol), ctypes.byref(st)))
    return st.as_dict()


class Batch:
    """A list of (X, C, assign, sums, counts) device-tensor tuples checked and marshalled once.

    ``run`` calls kmeans_run_batched on it as often as needed; the tensors are
    referenced, not copied, so their contents may change between runs (their
    shapes, dtypes and storage must not).
    """

    def __init__(self, problems):
        self.problems = list(problems)
        self.count = len(self.problems)
        self.arr = (Instance * self.count)()
        for b, (X, C, assign, sums, counts) in enumerate(self.problems):
            n, d, k = _check_tensors(X, C, assign, sums, counts)
            self.arr[b] = Instance(X.data_ptr(), n, d, k, C.data_ptr(), assign.data_ptr(), sums.data_ptr(),
                                   counts.data_ptr())
        self.stats = (Stats * self.count)()

    def run(self, iters, tol=0.0, *, precision="bf16", recheck=True, stream=None, warm_start=False,
            profile=False):
        """Runs the batch; returns the per-instance stats as a numpy structured array."""
        import numpy as np

        o = make_opts(precision, recheck, _stream_handle(stream), profile, warm_start)
        _check(_lib.kmeans_run_batched(ctypes.byref(o), self.arr, self.count, int(iters), float(tol), self.stats))
        return np.ctypeslib.as_array(self.stats).copy()


def run_batched(problems, iters, tol=0.0, *, precision="bf16", recheck=True, stream=None, warm_start=False,
                profile=False):
    """kmeans_run_batched over a list of (X, C, assign, sums, counts) device-tensor tuples (or a Batch).

    Every C is updated in place. Returns the list of per-instance stats dicts
    (with ``profile``, each carries the batch's device time per stage).
    """
    batch = problems if isinstance(problems, Batch) else Batch(problems)
    batch.run(iters, tol, precision=precision, recheck=recheck, stream=stream, warm_start=warm_start,
              profile=profile)
    return [s.as_dict() for s in batch.stats]


def _check_labelled(X, y, ncls):
    import torch

    if not (X.is_cuda and y.is_cuda):
        raise ValueError("X and y must be CUDA tensors")
    if X.dtype != torch.float32 or X.dim() != 2 or not X.is_contiguous():
        raise ValueError("X must be a contiguous float32 (n, d) tensor")
    n, d = X.shape
    if y.dtype != torch.int32 or tuple(y.shape) != (n,) or not y.is_contiguous():
        raise ValueError(f"y must be a contiguous int32 tensor of shape ({n},)")
    if ncls < 1:
        raise ValueError("ncls must be >= 1")
    return n, d


def gda_train(X, y, ncls, *, stream=None):
    """kmeans_gda_train: (phi [ncls], mu [ncls, d], sigma [d, d]) as float32 device tensors."""
    import torch

    n, d = _check_labelled(X, y, ncls)
    phi = torch.empty(ncls, dtype=torch.float32, device=X.device)
    mu = torch.empty(ncls, d, dtype=torch.float32, device=X.device)
    sigma = torch.empty(d, d, dtype=torch.float32, device=X.device)
    o = make_opts(stream=_stream_handle(stream))
    _check(_lib.kmeans_gda_train(ctypes.byref(o), X.data_ptr(), n, d, y.data_ptr(), int(ncls), phi.data_ptr(),
                                 mu.data_ptr(), sigma.data_ptr()))
    return phi, mu, sigma


def nb_train(X, y, ncls, *, stream=None):
    """kmeans_nb_train: (prior [ncls], theta [ncls, d]) as float32 device tensors."""
    import torch

    n, d = _check_labelled(X, y, ncls)
    prior = torch.empty(ncls, dtype=torch.float32, device=X.device)
    theta = torch.empty(ncls, d, dtype=torch.float32, device=X.device)
    o = make_opts(stream=_stream_handle(stream))
    _check(_lib.kmeans_nb_train(ctypes.byref(o), X.data_ptr(), n, d, y.data_ptr(), int(ncls), prior.data_ptr(),
                                theta.data_ptr()))
    return prior, theta


def spade_densities(X, apprx_width: float, kernel_width: float, *, policy: str = "last", stream=None):
    """kmeans_spade_densities: (densities int32 [n], counts int32 [n] (-1: skipped row),
    processed uint8 [n], stats dict) for the rows of a CUDA float32 (n, d) tensor."""
    import torch

    if not X.is_cuda or X.dtype != torch.float32 or X.dim() != 2 or not X.is_contiguous():
        raise ValueError("X must be a contiguous float32 (n, d) CUDA tensor")
    n, d = X.shape
    dens = torch.empty(n, dtype=torch.int32, device=X.device)
    counts = torch.empty(n, dtype=torch.int32, device=X.device)
    proc = torch.empty(n, dtype=torch.uint8, device=X.device)
    o = make_opts(stream=_stream_handle(stream))
    st = SpadeStats()
    _check(_lib.kmeans_spade_densities(ctypes.byref(o), X.data_ptr(), n, d, float(apprx_width), float(kernel_width),
                                       SPADE_POLICY[policy], dens.data_ptr(), counts.data_ptr(), proc.data_ptr(),
                                       ctypes.byref(st)))
    return dens, counts, proc, st.as_dict()


def version() -> int:
    return int(_lib.kmeans_version())


# ----------------------------------------------------------------------------- sharded step

def partials_len(k: int, d: int) -> int:
    """Entries of a partials buffer (KM_PARTIALS_LEN): k*d sums, k counts, objective, n_changed."""
    return k * d + k + 2


def step_partial(X, C, assign, part, *, precision="fp32", recheck=True, stream=None, warm_start=False,
                 deterministic=False, reuse_x=False, profile=False) -> dict:
    """A shard's part of a Lloyd step (kmeans_step_partial): assign is written, C is left alone, and
    ``part`` (float64, partials_len(k, d)) receives the shard's sums, counts, objective and n_changed."""
    import torch

    n, d = X.shape
    k = C.shape[0]
    for name, t, dt, shape in (("X", X, torch.float32, (n, d)), ("C", C, torch.float32, (k, d)),
                               ("assign", assign, torch.int32, (n,)),
                               ("part", part, torch.float64, (partials_len(k, d),))):
        if not t.is_cuda or t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor of shape {shape}")
    o = make_opts(precision, recheck, _stream_handle(stream), profile, warm_start, deterministic, reuse_x)
    st = Stats()
    _check(_lib.kmeans_step_partial(ctypes.byref(o), X.data_ptr(), n, d, C.data_ptr(), k, assign.data_ptr(),
                                    part.data_ptr(), ctypes.byref(st)))
    return st.as_dict()


def apply_partials(part, C, sums=None, counts=None, *, stream=None) -> dict:
    """The divide of a sharded step from a reduced partials buffer (kmeans_apply_partials); C is
    updated in place, sums / counts (optional) filled. Returns objective, n_changed, shift, n_empty."""
    import torch

    k, d = C.shape
    if not part.is_cuda or part.dtype != torch.float64 or part.numel() != partials_len(k, d) or not part.is_contiguous():
        raise ValueError("part must be a contiguous CUDA float64 tensor of partials_len(k, d) entries")
    o = make_opts(stream=_stream_handle(stream))
    st = Stats()
    _check(_lib.kmeans_apply_partials(ctypes.byref(o), part.data_ptr(), k, d, C.data_ptr(),
                                      sums.data_ptr() if sums is not None else None,
                                      counts.data_ptr() if counts is not None else None, ctypes.byref(st)))
    return st.as_dict()


# ----------------------------------------------------------------------------- diagnostics

def probe_mma(A, B, *, precision="bf16", stream=None):
    """D = A B^T (128 x 128, FP32) as the tensor core accumulates it (kmeans_probe_mma).

    A, B: contiguous CUDA tensors of shape (128, K): torch.bfloat16 for ``bf16``,
    torch.float8_e4m3fn (or uint8 bit patterns) for ``fp8``.
    """
    import torch

    for name, t in (("A", A), ("B", B)):
        if not t.is_cuda or not t.is_contiguous() or t.dim() != 2 or t.shape[0] != 128:
            raise ValueError(f"{name} must be a contiguous CUDA tensor of shape (128, K)")
    if A.shape != B.shape or A.dtype != B.dtype:
        raise ValueError("A and B must have the same shape and dtype")
    D = torch.empty(128, 128, dtype=torch.float32, device=A.device)
    _check(_lib.kmeans_probe_mma(PRECISION[precision], A.data_ptr(), B.data_ptr(), int(A.shape[1]), D.data_ptr(),
                                 _stream_handle(stream)))
    return D


def probe_ffma(iters=1 << 15, *, packed=True, stream=None):
    """(flops, ms) of one device-wide launch of independent FP32 FMA chains (kmeans_probe_ffma)."""
    fl = ctypes.c_double()
    ms = ctypes.c_float()
    _check(_lib.kmeans_probe_ffma(1 if packed else 0, int(iters), ctypes.byref(fl), ctypes.byref(ms),
                                  _stream_handle(stream)))
    return fl.value, ms.value
