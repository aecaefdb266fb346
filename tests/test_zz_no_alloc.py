"""kmeans_reduce_noalloc, the allocation-free keyed reduce, checked on the GPU.

Some callers cannot let a library allocate device memory: a host framework that
owns every byte of it (a serving runtime with a fixed budget, a plugin inside
another runtime), or code on a latency-critical path that must not pay for
cudaFree's device-wide synchronisation. kmeans_reduce_noalloc serves them: its
scratch is one fixed static device array. These tests call it through the C ABI
and compare each call's counts, sums and objective with

* the FP64 oracle's update and objective for the same assignment, and
* what the regular entry point kmeans_step_ex (cudaMalloc'd workspace) returns,

on two calls in a row (the second reuses the array the first one left behind),
at the array's size limits, after a call rejected for a bad label, and for
sizes beyond the limits. The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SUM_TOL = parity.CENTROID_TOL        # relative to the cluster's mean |x_it| times its count
OBJECTIVE_TOL = parity.OBJECTIVE_TOL  # relative


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans

    return kmeans


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


def _check_against_oracle(ref, X, C, assign, sums, counts, J):
    """Counts exact, sums within SUM_TOL (per cluster, relative to the members' mean |x| times the
    count), J within OBJECTIVE_TOL of the oracle's FP64 values for the same assignment."""
    Xh = X.cpu().numpy()
    Ch = C.cpu().numpy().astype(np.float64)
    a = assign.cpu().numpy()
    sums_ref, counts_ref, _ = ref.update(Xh, a, Ch)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), counts_ref), "counts differ from the oracle"
    scale, cnt = parity.member_scale(Xh, a, Ch.shape[0])
    err = np.abs(sums.cpu().numpy().astype(np.float64) - sums_ref).max(axis=1)
    assert np.all(err <= SUM_TOL * scale * np.maximum(cnt, 1) + 1e-30), "sums differ from the oracle"
    J_ref = ref.objective(Xh, Ch, a)
    assert abs(J - J_ref) <= OBJECTIVE_TOL * abs(J_ref), (J, J_ref)


def _check_against_regular(X, assign, sums, counts, J, sums_ref, counts_ref, J_ref):
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


def _one(km, ref, seed, n, d, k):
    X, C = _problem(seed, n, d, k)
    X, C = X.cuda(), C.cuda()
    assign, sums_ref, counts_ref, J_ref = _regular_step(km, X, C)
    rc, sums, counts, J = _noalloc(km, X, C, assign)
    assert rc == km.KM_OK, km.lib().kmeans_last_error()
    _check_against_oracle(ref, X, C, assign, sums, counts, J)
    _check_against_regular(X, assign, sums, counts, J, sums_ref, counts_ref, J_ref)


def test_noalloc_reduce_two_calls_in_a_row(km, ref):
    """Two different problems back to back: the second call starts from what the first left in
    the shared scratch array."""
    for seed, (n, d, k) in ((1, (200_000, 64, 256)), (2, (70_001, 33, 1000))):
        _one(km, ref, seed, n, d, k)


def test_noalloc_reduce_at_its_limits(km, ref):
    """n = 1,048,576, k = 8192, k * d = 262,144: every region of the scratch array fully used."""
    _one(km, ref, 3, 1 << 20, 32, 8192)


def test_noalloc_bad_label_then_valid_call(km, ref):
    """A label equal to k is rejected with KM_EINVAL (the device-side check stops the later
    stages); the next call, on the same array, clears that state and is correct."""
    X, C = _problem(4, 50_000, 24, 300)
    X, C = X.cuda(), C.cuda()
    assign, _, _, _ = _regular_step(km, X, C)
    bad = assign.clone()
    bad[12345] = 300
    rc, *_ = _noalloc(km, X, C, bad)
    assert rc == km.KM_EINVAL
    assert b"outside [0, k)" in km.lib().kmeans_last_error()
    _one(km, ref, 4, 50_000, 24, 300)


def test_noalloc_rejects_sizes_beyond_its_limit(km):
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
