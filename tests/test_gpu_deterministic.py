"""Deterministic reduce, reuse of cached codes across calls, and the one-device
form of the sharded step, through the C ABI.

* opts.deterministic: two runs from the same inputs return identical bits
  (centroids, sums, counts, labels, objective) in every precision, and every
  step keeps parity with the FP64 oracle (teacher forcing, the tolerances of
  tests/parity.py).
* opts.reuse_x: a sequence of one-step calls that reuses the previous call's
  codes and sorted order runs exactly like one kmeans_run (bitwise, with the
  deterministic reduce so that the comparison is exact).
* kmeans_step_partial + kmeans_apply_partials on one device (no exchange) give
  the same bits as kmeans_step_ex with the deterministic reduce.
"""
import numpy as np
import pytest

import parity
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"

CASES = [("fp32", 300_000, 64, 256), ("bf16", 400_000, 128, 512), ("fp8", 300_000, 96, 300),
         ("bf16x3", 100_000, 40, 100), ("fp32", 50_001, 200, 77), ("bf16", 70_001, 256, 130)]


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans

    return kmeans


def _data(n, d, k, seed=0):
    X = synth.mixture(9100 + seed + n % 97 + d + k, n, d, k, 10.0, 1.0)
    return torch.from_numpy(X).to(DEV), torch.from_numpy(X[:k].copy()).to(DEV), X


def _run(km, Xd, C0, iters, precision, **kw):
    C = C0.clone()
    out = km.run(Xd, C, iters, precision=precision, **kw)
    return C, out


@pytest.mark.parametrize("precision,n,d,k", CASES)
def test_deterministic_runs_are_bit_identical(km, precision, n, d, k):
    Xd, C0, _ = _data(n, d, k)
    C1, o1 = _run(km, Xd, C0, 8, precision, deterministic=True)
    C2, o2 = _run(km, Xd, C0, 8, precision, deterministic=True)
    assert torch.equal(C1, C2)
    assert torch.equal(o1.assign, o2.assign)
    assert torch.equal(o1.sums, o2.sums)
    assert torch.equal(o1.counts, o2.counts)
    assert o1.stats["objective"] == o2.stats["objective"]
    assert o1.stats["iters_done"] == 8


@pytest.mark.parametrize("precision,n,d,k", CASES)
def test_deterministic_steps_keep_parity(km, ref, precision, n, d, k):
    Xd, C0, X = _data(n, d, k, seed=1)
    Cd = C0.clone()
    a, s, c = km.alloc_outputs(Xd, Cd)
    near = 0
    for it in range(3):
        C_in = Cd.cpu().numpy().astype(np.float64)
        out = km.step(Xd, Cd, a, s, c, precision=precision, warm_start=it > 0, deterministic=True)
        ag = out.assign.cpu().numpy()
        m, _ = parity.check_assign(ref, X, C_in, ag)
        near += m
        parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), out.sums.cpu().numpy(), out.counts.cpu().numpy())
        parity.check_objective(ref, X, C_in, ag, out.stats["objective"])
    assert near <= max(2, n // 20000)


@pytest.mark.parametrize("precision,n,d,k", CASES[:4])
def test_reused_codes_steps_equal_one_run(km, precision, n, d, k):
    """Six one-step calls, the later ones with reuse_x (and warm_start), against kmeans_run(6)."""
    Xd, C0, _ = _data(n, d, k, seed=2)
    Cr, orun = _run(km, Xd, C0, 6, precision, deterministic=True)
    Cs = C0.clone()
    a, s, c = km.alloc_outputs(Xd, Cs)
    for it in range(6):
        st = km.step(Xd, Cs, a, s, c, precision=precision, deterministic=True, warm_start=it > 0,
                     reuse_x=it > 0).stats
    assert torch.equal(Cs, Cr)
    assert torch.equal(a, orun.assign)
    assert torch.equal(s, orun.sums)
    assert torch.equal(c, orun.counts)
    assert st["objective"] == orun.stats["objective"]
    assert st["n_changed"] == orun.stats["n_changed"]


def test_reuse_is_ignored_when_x_changes(km, ref):
    """reuse_x with a different X (or shape) than the cached call falls back to recomputing."""
    Xd, C0, X = _data(60_000, 64, 128, seed=3)
    Yd, _, Y = _data(60_000, 64, 128, seed=4)
    C = C0.clone()
    km.step(Xd, C, precision="bf16")
    C_in = C.cpu().numpy().astype(np.float64)
    out = km.step(Yd, C, precision="bf16", reuse_x=True)
    parity.check_assign(ref, Y, C_in, out.assign.cpu().numpy())
    parity.check_update(ref, Y, C_in, out.assign.cpu().numpy(), C.cpu().numpy(), out.sums.cpu().numpy(),
                        out.counts.cpu().numpy())


@pytest.mark.parametrize("precision,n,d,k", CASES[:4])
def test_partial_then_apply_equals_step(km, precision, n, d, k):
    Xd, C0, _ = _data(n, d, k, seed=5)
    Cs = C0.clone()
    o = km.step(Xd, Cs, precision=precision, deterministic=True)
    Cp = C0.clone()
    a = torch.zeros(n, dtype=torch.int32, device=DEV)
    part = torch.empty(km.partials_len(k, d), dtype=torch.float64, device=DEV)
    ps = km.step_partial(Xd, Cp, a, part, precision=precision, deterministic=True)
    assert torch.equal(Cp, C0), "a partial step must leave C alone"
    sums = torch.empty(k, d, dtype=torch.float32, device=DEV)
    counts = torch.empty(k, dtype=torch.int32, device=DEV)
    st = km.apply_partials(part, Cp, sums, counts)
    assert torch.equal(a, o.assign)
    assert torch.equal(Cp, Cs)
    assert torch.equal(sums, o.sums)
    assert torch.equal(counts, o.counts)
    assert st["objective"] == o.stats["objective"]
    assert st["n_changed"] == n and ps["n_changed"] == n
    assert st["n_empty"] == o.stats["n_empty"]
    assert abs(st["shift"] - o.stats["shift"]) <= 1e-12 * max(o.stats["shift"], 1.0)
    assert part[k * d: k * d + k].sum().item() == n


def test_apply_partials_rejects_bad_counts(km):
    k, d = 5, 3
    part = torch.zeros(km.partials_len(k, d), dtype=torch.float64, device=DEV)
    part[k * d + 2] = 1.5
    C = torch.ones(k, d, device=DEV)
    with pytest.raises(km.KMeansError) as e:
        km.apply_partials(part, C)
    assert e.value.status == km.KM_EINVAL
    assert torch.equal(C, torch.ones(k, d, device=DEV))


def test_batched_rejects_deterministic(km):
    Xd, C0, _ = _data(2000, 8, 4, seed=6)
    a, s, c = km.alloc_outputs(Xd, C0)
    o = km.make_opts("bf16", deterministic=True)
    arr = (km.Instance * 1)()
    arr[0] = km.Instance(Xd.data_ptr(), 2000, 8, 4, C0.data_ptr(), a.data_ptr(), s.data_ptr(), c.data_ptr())
    st = (km.Stats * 1)()
    import ctypes

    rc = km.lib().kmeans_run_batched(ctypes.byref(o), arr, 1, 2, 0.0, st)
    assert rc == km.KM_EUNSUPPORTED


@pytest.mark.parametrize("precision,n,d,k", CASES[:4])
def test_partial_then_apply_parity_default_reduce(km, ref, precision, n, d, k):
    """With the default (Kahan + FP64 atomics) reduce the partials hold the FP64 sums the segmented
    sum accumulates; the applied step keeps parity with the oracle."""
    Xd, C0, X = _data(n, d, k, seed=7)
    C = C0.clone()
    a = torch.zeros(n, dtype=torch.int32, device=DEV)
    part = torch.full((km.partials_len(k, d),), float("nan"), dtype=torch.float64, device=DEV)
    for it in range(2):
        C_in = C.cpu().numpy().astype(np.float64)
        km.step_partial(Xd, C, a, part, precision=precision, warm_start=it > 0, reuse_x=it > 0)
        sums = torch.empty(k, d, dtype=torch.float32, device=DEV)
        counts = torch.empty(k, dtype=torch.int32, device=DEV)
        st = km.apply_partials(part, C, sums, counts)
        ag = a.cpu().numpy()
        parity.check_assign(ref, X, C_in, ag)
        parity.check_update(ref, X, C_in, ag, C.cpu().numpy(), sums.cpu().numpy(), counts.cpu().numpy())
        parity.check_objective(ref, X, C_in, ag, st["objective"])
