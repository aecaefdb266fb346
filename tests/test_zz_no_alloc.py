"""kmeans_reduce_noalloc, the allocation-free keyed reduce, against the regular entry point.

Callers that may not allocate device memory (a host framework that owns all of
it, code that must not trigger cudaFree's device-wide synchronisation) use
kmeans_reduce_noalloc, whose scratch is a fixed static device array. This test
calls it through the C ABI twice in a row, on two different problems, and checks
each call's counts, sums and objective against what kmeans_step_ex (which uses
the regular cudaMalloc'd workspace) returns for the same assignment. The file is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SUM_TOL = 1e-5        # relative to the cluster's mean |x_it| times its count
OBJECTIVE_TOL = 1e-6  # relative


def _problem(seed, n, d, k):
    g = torch.Generator().manual_seed(seed)
    means = (torch.rand(k, d, generator=g) * 20 - 10)
    comp = torch.randint(0, k, (n,), generator=g)
    X = (means[comp] + torch.randn(n, d, generator=g)).contiguous()
    return X, X[:k].clone()


def _regular_step(km, X, C):
    """kmeans_step_ex: assignment, sums, counts and J(a, C) with the workspace entry point."""
    Cd = C.clone()
    out = km.step(X, Cd)
    return out.assign, out.sums, out.counts, out.stats["objective"]


def _noalloc(km, X, C, assign):
    n, d = X.shape
    k = C.shape[0]
    sums = torch.empty(k, d, dtype=torch.float32, device=X.device)
    counts = torch.empty(k, dtype=torch.int32, device=X.device)
    obj = ctypes.c_double(0.0)
    rc = km.lib().kmeans_reduce_noalloc(X.data_ptr(), n, d, C.data_ptr(), k, assign.data_ptr(),
                                        sums.data_ptr(), counts.data_ptr(), ctypes.byref(obj), None)
    return rc, sums, counts, obj.value


def _compare(X, assign, sums, counts, J, sums_ref, counts_ref, J_ref):
    assert torch.equal(counts, counts_ref)
    a = assign.long()
    k = counts.shape[0]
    absmean = torch.zeros(k, X.shape[1], dtype=torch.float64, device=X.device)
    absmean.index_add_(0, a, X.abs().double())
    cnt = counts.double().clamp(min=1)
    scale = (absmean / cnt[:, None]).max(dim=1).values * cnt
    err = (sums.double() - sums_ref.double()).abs().max(dim=1).values
    assert torch.all(err <= SUM_TOL * scale + 1e-30), float((err / scale.clamp(min=1e-30)).max())
    assert abs(J - J_ref) <= OBJECTIVE_TOL * abs(J_ref)


def test_noalloc_reduce_matches_regular_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans as km

    for seed, (n, d, k) in ((1, (200_000, 64, 256)), (2, (70_001, 33, 1000))):
        X, C = _problem(seed, n, d, k)
        X, C = X.cuda(), C.cuda()
        assign, sums_ref, counts_ref, J_ref = _regular_step(km, X, C)
        rc, sums, counts, J = _noalloc(km, X, C, assign)
        assert rc == km.KM_OK, km.lib().kmeans_last_error()
        _compare(X, assign, sums, counts, J, sums_ref, counts_ref, J_ref)


def test_noalloc_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans as km

    X = torch.zeros(16, 300, device="cuda")  # d = 300 > 256
    C = torch.zeros(2, 300, device="cuda")
    a = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc, *_ = _noalloc(km, X, C, a)
    assert rc == km.KM_EINVAL
    X = torch.zeros(2, 200, device="cuda")  # k * d = 2000 * 200 > 262144 (never touched: rejected first)
    big_k = 2000
    rc = km.lib().kmeans_reduce_noalloc(X.data_ptr(), 2, 200, X.data_ptr(), big_k, a.data_ptr(), X.data_ptr(),
                                        a.data_ptr(), None, None)
    assert rc == km.KM_EINVAL
    assert b"no-allocation limit" in km.lib().kmeans_last_error()
