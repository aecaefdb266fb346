"""GPU parity of the fused Lloyd step against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import parity
import synth
from synth import WORKLOADS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans

    return kmeans


DEV = "cuda:0"


def gpu_steps(km, orc, X, C0, steps, precision="fp32", rows=None, warm=True):
    """Teacher-forced per-step parity; returns the number of near-tie mismatches and the stats.

    With ``warm`` every step after the first passes the previous step's assignment in
    (warm_start), as the steps of a run do."""
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(np.ascontiguousarray(C0, dtype=np.float32)).to(DEV)
    assign, sums, counts = km.alloc_outputs(Xd, Cd)
    near = 0
    stats = []
    for it in range(steps):
        C_in = Cd.cpu().numpy().astype(np.float64)
        out = km.step(Xd, Cd, assign, sums, counts, precision=precision, warm_start=warm and it > 0)
        a = out.assign.cpu().numpy()
        m, _ = parity.check_assign(orc, X, C_in, a, rows=rows)
        near += m
        parity.check_update(orc, X, C_in, a, Cd.cpu().numpy(), out.sums.cpu().numpy(), out.counts.cpu().numpy())
        parity.check_objective(orc, X, C_in, a, out.stats["objective"])
        assert out.stats["iters_done"] == 1
        stats.append(out.stats)
    return near, stats


def test_plain_workload_all_iterations(km, ref):
    w = WORKLOADS["plain_n10k_d16_k8"]
    X, C0 = synth.workload_data(w)
    near, stats = gpu_steps(km, ref, X, C0, w.iters)
    assert stats[0]["n_changed"] == w.n
    assert near <= 2


@pytest.mark.parametrize("n,d,k", [
    (1, 1, 1), (5, 3, 5), (7, 1, 2), (1000, 1, 7), (129, 2, 128), (4099, 33, 130),
    (2000, 17, 129), (3000, 256, 20), (1500, 255, 300), (20037, 64, 256), (513, 96, 511),
])
def test_shapes_ragged(km, ref, n, d, k):
    X = synth.mixture(1000 + n + d + k, n, d, max(k, 1), 5.0, 1.0)
    near, _ = gpu_steps(km, ref, X, X[:k].copy(), 3)
    assert near <= max(2, n // 1000)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("n,d,k", [(3000, 64, 256), (2100, 20, 70)])
def test_rows_not_16_byte_aligned(km, ref, precision, n, d, k):
    """X and C starting 4 bytes past a 16-byte boundary (contiguous views one float into a
    buffer): every kernel that reads them in 16-byte pieces must fall back to 4-byte ones, so
    any float-aligned X and C give the same parity."""
    X = synth.mixture(5150 + n + d, n, d, k, 5.0, 1.0)
    buf = torch.zeros(n * d + 1, dtype=torch.float32, device=DEV)
    Xd = buf[1:].view(n, d)
    Xd.copy_(torch.from_numpy(X))
    assert Xd.is_contiguous() and Xd.data_ptr() % 16 == 4
    cbuf = torch.zeros(k * d + 1, dtype=torch.float32, device=DEV)
    Cd = cbuf[1:].view(k, d)
    Cd.copy_(torch.from_numpy(X[:k].copy()))
    assert Cd.is_contiguous() and Cd.data_ptr() % 16 == 4
    assign, sums, counts = km.alloc_outputs(Xd, Cd)
    for it in range(2):
        C_in = Cd.cpu().numpy().astype(np.float64)
        out = km.step(Xd, Cd, assign, sums, counts, precision=precision, warm_start=it > 0)
        a = out.assign.cpu().numpy()
        near, _ = parity.check_assign(ref, X, C_in, a)
        assert near <= 2
        parity.check_update(ref, X, C_in, a, Cd.cpu().numpy(), out.sums.cpu().numpy(), out.counts.cpu().numpy())


def test_k_equals_one_and_n(km, ref):
    X = synth.mixture(77, 700, 9, 3, 4.0, 1.0)
    gpu_steps(km, ref, X, X[:1].copy(), 2)
    # k = n with distinct points and C0 = X: identity assignment, nothing moves
    Xd = torch.from_numpy(X).to(DEV)
    Cd = Xd.clone()
    out = km.step(Xd, Cd)
    assert np.array_equal(out.assign.cpu().numpy(), np.arange(700, dtype=np.int32))
    assert torch.equal(Cd, Xd)
    assert out.stats["objective"] == 0.0


def test_exact_ties_and_empty_clusters(km, ref):
    # integer data with duplicated centroids: exact ties must go to the lowest index and the
    # duplicates must stay empty with their centroid unchanged
    rng = np.random.default_rng(5)
    X = rng.integers(-4, 5, size=(5000, 3)).astype(np.float32)
    C0 = np.concatenate([X[:6], X[:6], X[6:10]])  # 6 duplicated pairs
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(C0).to(DEV)
    out = km.step(Xd, Cd)
    a = out.assign.cpu().numpy()
    ra, *_ = ref.assign(X, C0.astype(np.float64))
    assert np.array_equal(a, ra), "exact ties must resolve to the lowest index"
    counts = out.counts.cpu().numpy()
    assert np.all(counts[6:12] == 0)
    assert np.array_equal(Cd.cpu().numpy()[6:12], C0[6:12])
    assert out.stats["n_empty"] >= 6
    parity.check_update(ref, X, C0.astype(np.float64), a, Cd.cpu().numpy(), out.sums.cpu().numpy(), counts)


def test_golden_examples_on_gpu(km):
    import oracle_pins

    for path in oracle_pins.golden_files():
        d, Xf, C0f, steps = oracle_pins.parse_golden(path)
        X = torch.tensor([float(v) for v in Xf], dtype=torch.float32, device=DEV).reshape(-1, d)
        C = torch.tensor([float(v) for v in C0f], dtype=torch.float32, device=DEV).reshape(-1, d)
        for exp in steps:
            out = km.step(X, C)
            assert out.assign.cpu().tolist() == exp["assign"], path
            assert out.counts.cpu().tolist() == exp["counts"], path
            assert np.allclose(C.cpu().numpy().ravel(), [float(v) for v in exp["C"]], rtol=2e-7, atol=0), path
            assert abs(out.stats["objective"] - float(exp["J"])) <= 1e-6 * max(1.0, float(exp["J"])), path


def test_run_matches_free_running_oracle(km, ref):
    w = WORKLOADS["plain_n10k_d16_k8"]
    X, C0 = synth.workload_data(w)
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(C0).to(DEV)
    out = km.run(Xd, Cd, w.iters)
    r = ref.run(X, C0.astype(np.float64), w.iters)
    assert out.stats["iters_done"] == w.iters
    a = out.assign.cpu().numpy()
    assert (a != r["assign"]).sum() <= 2
    assert abs(out.stats["objective"] - r["objectives"][-1]) <= 1e-5 * r["objectives"][-1]
    scale, _ = parity.member_scale(X, r["assign"], w.k)
    assert np.all(np.abs(Cd.cpu().numpy() - r["C"]).max(axis=1) <= 1e-5 * scale + 1e-6)


def test_run_graph_replay_and_resume(km, ref):
    X = synth.mixture(31, 6000, 12, 10, 6.0, 1.0)
    Xd = torch.from_numpy(X).to(DEV)
    C0 = torch.from_numpy(X[:10].copy()).to(DEV)
    C1 = C0.clone()
    o1 = km.run(Xd, C1, 8)
    # same call again replays the cached graph and must give the same result
    C2 = C0.clone()
    a2, s2, c2 = km.alloc_outputs(Xd, C2)
    o2 = km.run(Xd, C2, 8, assign=a2, sums=s2, counts=c2)
    C3 = C0.clone()
    o3 = km.run(Xd, C3, 8, assign=a2, sums=s2, counts=c2)  # identical pointers: cached graph
    # the segmented sums add FP64 partials in no set order, so centroids may differ in the last ulp
    assert (o2.assign != o3.assign).sum().item() <= 2
    assert torch.allclose(C2, C3, rtol=1e-6, atol=1e-6)
    # 4 + 4 steps reach the state of 8 steps (C is the whole state)
    C4 = C0.clone()
    km.run(Xd, C4, 4)
    o4 = km.run(Xd, C4, 4)
    assert (o4.assign != o1.assign).sum().item() <= 2
    assert torch.allclose(C4, C1, rtol=0, atol=1e-4)


def test_assignment_is_deterministic(km):
    # the assignment of a step depends only on X and C, never on reduction order
    X = synth.mixture(13, 20000, 40, 64, 5.0, 1.0)
    Xd = torch.from_numpy(X).to(DEV)
    C0 = torch.from_numpy(X[:64].copy()).to(DEV)
    outs = [km.step(Xd, C0.clone()) for _ in range(3)]
    for o in outs[1:]:
        assert torch.equal(o.assign, outs[0].assign)
        assert torch.equal(o.counts, outs[0].counts)


def test_stop_rule(km, ref):
    X = synth.mixture(9, 4000, 5, 4, 30.0, 0.5)  # well separated: converges in a few steps
    Xd = torch.from_numpy(X).to(DEV)
    C = torch.from_numpy(X[:4].copy()).to(DEV)
    out = km.run(Xd, C, 50, tol=1e-300)
    r = ref.run(X, X[:4].astype(np.float64), 50, tol=1e-300)
    assert out.stats["iters_done"] == r["iters_done"] < 50
    assert out.stats["n_changed"] == 0


def test_permutation_equivariance(km):
    X = synth.mixture(12, 5000, 20, 16, 5.0, 1.0)
    perm = np.random.default_rng(0).permutation(5000)
    C0 = torch.from_numpy(X[:16].copy()).to(DEV)
    o1 = km.step(torch.from_numpy(X).to(DEV), C0.clone())
    o2 = km.step(torch.from_numpy(np.ascontiguousarray(X[perm])).to(DEV), C0.clone())
    assert np.array_equal(o2.assign.cpu().numpy(), o1.assign.cpu().numpy()[perm])
    assert torch.equal(o1.counts, o2.counts)


def test_host_entry_point(km, ref):
    X = synth.mixture(44, 9000, 24, 30, 8.0, 1.0)
    C0 = X[:30].copy()
    Ch = C0.copy()
    a = np.empty(9000, np.int32)
    s = np.empty((30, 24), np.float32)
    c = np.empty(30, np.int32)
    st = km.run_host(X, Ch, 5, 0.0, a, s, c)
    Cd = torch.from_numpy(C0).to(DEV)
    out = km.run(torch.from_numpy(X).to(DEV), Cd, 5)
    assert st["iters_done"] == 5
    assert (a != out.assign.cpu().numpy()).sum() <= 2
    assert np.allclose(Ch, Cd.cpu().numpy(), rtol=0, atol=1e-4)
    assert c.sum() == 9000


def test_errors(km):
    X = torch.randn(100, 4, device=DEV)
    C = X[:5].clone()
    a, s, c = km.alloc_outputs(X, C)
    # a host array through the device entry point is rejected by the C ABI itself
    import ctypes

    Xh = np.zeros((100, 4), np.float32)
    st = km.Stats()
    rc = km.lib().kmeans_step_ex(None, Xh.ctypes.data, 100, 4, C.data_ptr(), 5, a.data_ptr(), s.data_ptr(),
                                 c.data_ptr(), ctypes.byref(st))
    assert rc == km.KM_EINVAL and b"device memory" in km.lib().kmeans_last_error()
    Xn = X.clone()
    Xn[17, 2] = float("nan")
    C_before = C.clone()
    with pytest.raises(km.KMeansError) as e:
        km.step(Xn, C, a, s, c)
    assert e.value.status == km.KM_ENONFINITE
    assert torch.equal(C, C_before), "C must hold its value on entry after an error"
    Cn = C.clone()
    Cn[1, 0] = float("inf")
    with pytest.raises(km.KMeansError) as e:
        km.step(X, Cn, a, s, c)
    assert e.value.status == km.KM_ENONFINITE
    # the library still works after the errors
    out = km.step(X, C, a, s, c)
    assert out.counts.sum().item() == 100


@pytest.mark.slow
def test_full_size_fp32_workload(km, ref):
    """The benchmark's launch configuration (kmeans_run, 20 graph-captured steps) at full size,
    checked by the O(nd) update in full and the O(nkd) assignment on a random sample of rows."""
    w = WORKLOADS["fp32_n1M_d64_k256"]
    X, C0 = synth.workload_data(w)
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(C0).to(DEV)
    out = km.run(Xd, Cd, w.iters)
    assert out.stats["iters_done"] == w.iters
    a20 = out.assign.cpu().numpy()
    C20 = Cd.cpu().numpy()
    counts = out.counts.cpu().numpy()
    assert counts.sum() == w.n and np.array_equal(counts, np.bincount(a20, minlength=w.k))
    # one more step from C^20: sampled argmin parity and the full update
    C_in = C20.astype(np.float64)
    o = km.step(Xd, Cd)
    a21 = o.assign.cpu().numpy()
    rows = np.sort(np.random.default_rng(1).choice(w.n, 8192, replace=False))
    parity.check_assign(ref, X, C_in, a21, rows=rows)
    parity.check_update(ref, X, C_in, a21, Cd.cpu().numpy(), o.sums.cpu().numpy(), o.counts.cpu().numpy())
    parity.check_objective(ref, X, C_in, a21, o.stats["objective"])
    assert o.stats["objective"] <= out.stats["objective"] * (1 + 1e-6)


# ----------------------------------------------------------------------------- tensor-core path

@pytest.mark.parametrize("precision", ["bf16", "fp8", "bf16x3"])
def test_tc_smoke(km, ref, precision):
    X = synth.mixture(5, 1000, 16, 8, 10.0, 1.0)
    near, stats = gpu_steps(km, ref, X, X[:8].copy(), 2, precision=precision)
    assert near <= 2


@pytest.mark.parametrize("precision", ["bf16", "fp8", "bf16x3"])
@pytest.mark.parametrize("n,d,k", [
    (1, 1, 1), (5, 3, 5), (129, 2, 128), (4099, 33, 130), (2000, 17, 129), (3000, 256, 20),
    (1500, 255, 300), (20037, 64, 256), (513, 96, 511), (700, 128, 700), (3333, 200, 1000),
])
def test_tc_shapes_ragged(km, ref, precision, n, d, k):
    X = synth.mixture(2000 + n + d + k, n, d, max(k, 1), 5.0, 1.0)
    near, stats = gpu_steps(km, ref, X, X[:k].copy(), 3, precision=precision)
    assert near <= max(2, n // 1000)


@pytest.mark.parametrize("precision", ["bf16", "fp8", "bf16x3"])
def test_tc_precision_workload_sample(km, ref, precision):
    """The first 65,536 points of the 4M x 128 x 1024 workload, 3 teacher-forced steps."""
    w = WORKLOADS["prec_n4M_d128_k1024"]
    X, C0 = synth.workload_data(w, rows=65536)
    near, stats = gpu_steps(km, ref, X, C0, 3, precision=precision)
    assert near <= 20
    assert all(s["n_flagged"] < 65536 for s in stats)


def test_split_bf16_margin_is_tighter(km, ref):
    """Two-part BF16 codes shrink the near-tie margin by about 2^-8 against BF16 (the
    residual terms drop from 2^-9 ||x|| ||c|| to the accumulation bound), so far fewer
    points are flagged on the same step; both assignments are exact."""
    w = WORKLOADS["prec_n4M_d128_k1024"]
    X, C0 = synth.workload_data(w, rows=65536)
    Xd = torch.from_numpy(X).to(DEV)
    flagged = {}
    for precision in ("bf16", "bf16x3"):
        Cd = torch.from_numpy(C0).to(DEV)
        out = km.step(Xd, Cd, precision=precision)
        parity.check_assign(ref, X, C0.astype(np.float64), out.assign.cpu().numpy())
        flagged[precision] = out.stats["n_flagged"]
    assert flagged["bf16"] > 1000
    assert flagged["bf16x3"] * 10 <= flagged["bf16"], flagged


@pytest.mark.slow
def test_tc_large_workload_sample(km, ref):
    """The first 16,384 points of the 8M x 256 x 8192 workload with FP8, 2 teacher-forced steps."""
    w = WORKLOADS["large_n8M_d256_k8192"]
    X, C0 = synth.workload_data(w, rows=16384)
    near, stats = gpu_steps(km, ref, X, C0, 2, precision="fp8")
    assert near <= 20


def _full_size_tc(km, ref, w, precision, sample):
    """kmeans_run of the workload's iterations at full size (the bench's launch configuration),
    then one more step from the result: the assignment on a random row sample, the O(nd)
    update and the objective in full."""
    X, C0 = synth.workload_data(w)
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(C0).to(DEV)
    out = km.run(Xd, Cd, w.iters, precision=precision)
    assert out.stats["iters_done"] == w.iters
    counts = out.counts.cpu().numpy()
    assert counts.sum() == w.n and np.array_equal(counts, np.bincount(out.assign.cpu().numpy(), minlength=w.k))
    C_in = Cd.cpu().numpy().astype(np.float64)
    o = km.step(Xd, Cd, out.assign, out.sums, out.counts, precision=precision, warm_start=True)
    a1 = o.assign.cpu().numpy()
    rows = np.sort(np.random.default_rng(7).choice(w.n, sample, replace=False))
    parity.check_assign(ref, X, C_in, a1, rows=rows)
    parity.check_update(ref, X, C_in, a1, Cd.cpu().numpy(), o.sums.cpu().numpy(), o.counts.cpu().numpy())
    parity.check_objective(ref, X, C_in, a1, o.stats["objective"])
    assert o.stats["objective"] <= out.stats["objective"] * (1 + 1e-6)


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["bf16", "fp8", "bf16x3"])
def test_full_size_precision_workload(km, ref, precision):
    _full_size_tc(km, ref, WORKLOADS["prec_n4M_d128_k1024"], precision, 8192)


@pytest.mark.slow
def test_full_size_large_workload(km, ref):
    _full_size_tc(km, ref, WORKLOADS["large_n8M_d256_k8192"], "fp8", 8192)  # sample >= k (oracle precondition)


@pytest.mark.parametrize("precision", ["bf16", "fp8", "bf16x3"])
def test_tc_run_matches_free_running_oracle(km, ref, precision):
    """Graph-captured runs (seeded from the second step on) against the free-running oracle."""
    X = synth.mixture(77, 30000, 48, 40, 8.0, 1.0)
    C0 = X[:40].copy()
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(C0).to(DEV)
    out = km.run(Xd, Cd, 8, precision=precision)
    r = ref.run(X, C0.astype(np.float64), 8)
    assert out.stats["iters_done"] == 8
    a = out.assign.cpu().numpy()
    assert (a != r["assign"]).sum() <= 3
    assert abs(out.stats["objective"] - r["objectives"][-1]) <= 1e-5 * r["objectives"][-1]


def test_warm_start_ignores_bad_labels(km, ref):
    X = synth.mixture(8, 3000, 24, 12, 6.0, 1.0)
    Xd = torch.from_numpy(X).to(DEV)
    for precision in ("fp32", "bf16", "fp8", "bf16x3"):
        Cd = torch.from_numpy(X[:12].copy()).to(DEV)
        a, s, c = km.alloc_outputs(Xd, Cd)
        a.copy_(torch.randint(-5, 20, (3000,), dtype=torch.int32))  # garbage, some out of range
        C_in = Cd.cpu().numpy().astype(np.float64)
        out = km.step(Xd, Cd, a, s, c, precision=precision, warm_start=True)
        parity.check_assign(ref, X, C_in, out.assign.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp8", "bf16"])
def test_queued_points_rescored(km, ref, precision):
    """Centroids duplicated nine times: every point has nine equal candidates (more than the eight
    slots), so it is queued, re-scored (E4M3 runs: BF16 codes on the tensor cores; BF16 runs: the
    FP32 slab kernel), still tied, and settled over all k with the lowest index."""
    n = 60000  # enough tied points that the full re-checks are queued rather than settled one by one
    X = synth.mixture(61, n, 64, 12, 6.0, 1.0)
    base = X[:12].copy()
    C0 = np.repeat(base, 9, axis=0)  # centroid 9 q + r is a copy of point q
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(C0).to(DEV)
    a, s, c = km.alloc_outputs(Xd, Cd)
    a.copy_(torch.from_numpy(np.zeros(n, np.int32)))
    out = km.step(Xd, Cd, a, s, c, precision=precision, warm_start=True)
    assert out.stats["n_full"] > 0
    ag = out.assign.cpu().numpy()
    parity.check_assign(ref, X, C0.astype(np.float64), ag)
    assert np.all(ag % 9 == 0)  # the lowest index of each tied group


def test_tc_recheck_off_still_runs(km):
    X = synth.mixture(3, 5000, 32, 20, 5.0, 1.0)
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(X[:20].copy()).to(DEV)
    out = km.step(Xd, Cd, precision="bf16", recheck=False)
    a = out.assign.cpu().numpy()
    assert a.min() >= 0 and a.max() < 20 and out.counts.sum().item() == 5000


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8", "bf16x3"])
def test_profiled_runs(km, ref, precision):
    """opts.profile records stage events inside the captured graph; results are unchanged."""
    X = synth.mixture(21, 20000, 64, 50, 8.0, 1.0)
    Xd = torch.from_numpy(X).to(DEV)
    C0 = torch.from_numpy(X[:50].copy()).to(DEV)
    for iters in (1, 5):
        C = C0.clone()
        out = km.run(Xd, C, iters, precision=precision, profile=True)
        st = out.stats["stage_ms"]
        assert st["assign"] > 0 and st["divide"] > 0 and st["xnorm"] > 0
        assert out.stats["iters_done"] == iters
    C = C0.clone()
    r = ref.run(X, X[:50].astype(np.float64), 5)
    assert (out.assign.cpu().numpy() != r["assign"]).sum() <= 3


@pytest.mark.parametrize("n,d,k", [(10000, 16, 8), (16384, 16, 32), (2048, 64, 64), (777, 3, 5), (4096, 33, 40),
                                   (5000, 8, 1)])
def test_small_problems_single_launch(km, ref, n, d, k):
    """Small FP32 problems (n <= 16384, k <= 64, d <= 64, n k d <= 2^23; the cases include both limits)
    run every step of a call in one kernel launch; each step keeps parity with the oracle (teacher
    forcing) and the result equals the staged path's (opts.profile forces it)."""
    X = synth.mixture(4400 + n + d + k, n, d, max(k, 2), 6.0, 1.0)
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(X[:k].copy()).to(DEV)
    a, s, c = km.alloc_outputs(Xd, Cd)
    for it in range(3):
        C_in = Cd.cpu().numpy().astype(np.float64)
        out = km.step(Xd, Cd, a, s, c, warm_start=it > 0)
        ag = out.assign.cpu().numpy()
        parity.check_assign(ref, X, C_in, ag)
        parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), out.sums.cpu().numpy(), out.counts.cpu().numpy())
        parity.check_objective(ref, X, C_in, ag, out.stats["objective"])
    C1 = torch.from_numpy(X[:k].copy()).to(DEV)
    o1 = km.run(Xd, C1, 6)
    assert o1.stats["launches"] == 1, o1.stats
    C2 = torch.from_numpy(X[:k].copy()).to(DEV)
    o2 = km.run(Xd, C2, 6, profile=True)
    assert o2.stats["launches"] > 6
    assert (o1.assign != o2.assign).sum().item() <= 2
    assert torch.allclose(C1, C2, rtol=1e-6, atol=1e-6)
    assert abs(o1.stats["objective"] - o2.stats["objective"]) <= 1e-6 * abs(o2.stats["objective"])


@pytest.mark.parametrize("n,d,k,tol", [(10000, 16, 8, 1e-4), (3000, 40, 64, 1e-3), (16384, 64, 8, 0.0)])
def test_small_problems_stop_rule_and_reproducible(km, n, d, k, tol):
    """The one-launch path stops after the same step as the staged path (tol > 0; tol = 0 runs every
    step), its last step's counts agree, and two calls return identical bits: each cluster's sum is
    taken in a fixed order whatever the scheduling."""
    X = synth.mixture(5100 + n + d + k, n, d, k, 6.0, 1.0)
    Xd = torch.from_numpy(X).to(DEV)
    outs = []
    for prof in (False, False, True):
        C = torch.from_numpy(X[:k].copy()).to(DEV)
        outs.append((C, km.run(Xd, C, 60, tol=tol, profile=prof)))
    (C1, o1), (C2, o2), (C3, o3) = outs
    assert o1.stats["launches"] == 1 and o3.stats["launches"] > 1
    assert o1.stats["iters_done"] == o3.stats["iters_done"]
    assert (o1.stats["iters_done"] < 60) == (tol > 0)
    assert o1.stats["n_changed"] == o3.stats["n_changed"]
    assert o1.stats["n_empty"] == o3.stats["n_empty"]
    assert torch.equal(C1, C2) and torch.equal(o1.assign, o2.assign) and torch.equal(o1.sums, o2.sums)
    assert torch.equal(o1.counts, o2.counts) and o1.stats["objective"] == o2.stats["objective"]
    assert torch.equal(o1.counts, o3.counts)
    assert torch.allclose(C1, C3, rtol=1e-6, atol=1e-6)
    assert abs(o1.stats["objective"] - o3.stats["objective"]) <= 1e-6 * abs(o3.stats["objective"])


@pytest.mark.parametrize("precision", ["bf16", "fp8", "bf16x3"])
def test_offset_data_centred_codes(km, ref, precision):
    """A common offset of 1000 in every coordinate: the quantised paths code x - mu and c - mu (mu =
    the mean of the call's initial centroids), so the margin is that of the centred data. Before
    centring, BF16 and E4M3 flagged every point (all-centroid re-checks); parity per step, and the
    flag rate stays that of the data without the offset."""
    n, d, k = 120_000, 64, 48
    X0 = synth.mixture(0xABD, n, d, k, 20.0, 1.0)
    rates = []
    for off in (0.0, 1000.0):
        X = (X0 + np.float32(off)).astype(np.float32)
        Xd = torch.from_numpy(X).to(DEV)
        Cd = torch.from_numpy(X[:k].copy()).to(DEV)
        a, s, c = km.alloc_outputs(Xd, Cd)
        for it in range(3):
            C_in = Cd.cpu().numpy().astype(np.float64)
            out = km.step(Xd, Cd, a, s, c, precision=precision, warm_start=it > 0)
            ag = out.assign.cpu().numpy()
            parity.check_assign(ref, X, C_in, ag)
            parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), out.sums.cpu().numpy(), out.counts.cpu().numpy())
            parity.check_objective(ref, X, C_in, ag, out.stats["objective"])
        rates.append((out.stats["n_flagged"] / n, out.stats["n_full"] / n))
    (f0, _), (f1, full1) = rates
    assert f1 <= f0 + 0.02 and full1 <= 0.01, rates
