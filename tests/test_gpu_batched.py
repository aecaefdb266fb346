"""Batched runs (kmeans_run_batched) against the FP64 oracle, instance by instance."""
import numpy as np
import pytest

import parity
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans

    return kmeans


SHAPES = [(1000, 8, 4), (5000, 32, 40), (3001, 64, 7), (2500, 128, 300), (129, 8, 129), (777, 17, 1),
          (4096, 64, 512), (10000, 32, 130), (600, 100, 60), (2048, 128, 64), (1500, 8, 100), (300, 1, 3)]


def make_batch(shapes, seed0=500):
    data = []
    for b, (n, d, k) in enumerate(shapes):
        X = synth.mixture(seed0 + b, n, d, max(k, 1), 10.0, 1.0)
        data.append((X, X[:k].copy()))
    return data


def to_device(km, data):
    probs = []
    for X, C0 in data:
        Xd = torch.from_numpy(X).to(DEV)
        Cd = torch.from_numpy(C0).to(DEV)
        a, s, c = km.alloc_outputs(Xd, Cd)
        probs.append((Xd, Cd, a, s, c))
    return probs


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_batched_single_step_parity(km, ref, precision):
    data = make_batch(SHAPES)
    probs = to_device(km, data)
    stats = km.run_batched(probs, 1, precision=precision)
    for (X, C0), (Xd, Cd, a, s, c), st in zip(data, probs, stats):
        C_in = C0.astype(np.float64)
        ag = a.cpu().numpy()
        parity.check_assign(ref, X, C_in, ag)
        parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), s.cpu().numpy(), c.cpu().numpy())
        parity.check_objective(ref, X, C_in, ag, st["objective"])
        assert st["iters_done"] == 1


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_batched_small_d_parity(km, ref, precision):
    """Rows of d <= 16 are packed several per warp step in the segmented sum (d = 1 ... 16,
    powers of two and not, mixed with unpacked instances)."""
    shapes = [(2000, 3, 9), (1111, 13, 20), (640, 16, 33), (800, 5, 6), (999, 2, 4), (1500, 24, 11), (700, 9, 70)]
    data = make_batch(shapes, seed0=4100)
    probs = to_device(km, data)
    stats = km.run_batched(probs, 2, precision=precision)
    # one more step from the result, checked against the oracle's step from the same centroids
    C_ins = [p[1].cpu().numpy().astype(np.float64) for p in probs]
    stats = km.run_batched(probs, 1, precision=precision, warm_start=True)
    for (X, _), (Xd, Cd, a, s, c), C_in, st in zip(data, probs, C_ins, stats):
        ag = a.cpu().numpy()
        parity.check_assign(ref, X, C_in, ag)
        parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), s.cpu().numpy(), c.cpu().numpy())
        parity.check_objective(ref, X, C_in, ag, st["objective"])


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_batched_warm_steps_parity(km, ref, precision):
    """Steps after the first pass the previous assignment in (warm start), one step per call."""
    data = make_batch(SHAPES, seed0=900)
    probs = to_device(km, data)
    km.run_batched(probs, 1, precision=precision)
    for _ in range(2):
        C_ins = [p[1].cpu().numpy().astype(np.float64) for p in probs]
        stats = km.run_batched(probs, 1, precision=precision, warm_start=True)
        for (X, _), (Xd, Cd, a, s, c), C_in, st in zip(data, probs, C_ins, stats):
            ag = a.cpu().numpy()
            parity.check_assign(ref, X, C_in, ag)
            parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), s.cpu().numpy(), c.cpu().numpy())


def test_batched_run_matches_free_running_oracle(km, ref):
    data = make_batch(SHAPES, seed0=1300)
    probs = to_device(km, data)
    stats = km.run_batched(probs, 6, precision="bf16")
    for (X, C0), (Xd, Cd, a, s, c), st in zip(data, probs, stats):
        r = ref.run(X, C0.astype(np.float64), 6)
        assert st["iters_done"] == 6
        ag = a.cpu().numpy()
        assert (ag != r["assign"]).sum() <= max(3, X.shape[0] // 500)
        assert abs(st["objective"] - r["objectives"][-1]) <= 1e-4 * max(r["objectives"][-1], 1e-12)


def test_batched_equals_single_instance_runs(km):
    """The batched graph and separate kmeans_run calls give the same assignments (up to near-ties)."""
    data = make_batch(SHAPES[:6], seed0=77)
    probs = to_device(km, data)
    km.run_batched(probs, 4, precision="bf16")
    for (X, C0), (Xd, Cd, a, s, c) in zip(data, probs):
        Cs = torch.from_numpy(C0).to(DEV)
        out = km.run(Xd, Cs, 4, precision="bf16")
        assert (out.assign != a).sum().item() <= max(2, X.shape[0] // 1000)
        assert torch.allclose(Cs, Cd, rtol=1e-4, atol=1e-4)


def test_batched_stop_rule_per_instance(km, ref):
    # well separated instances converge at different steps; each stops on its own
    shapes = [(2000, 4, 3), (3000, 8, 5), (1500, 16, 2)]
    data = []
    for b, (n, d, k) in enumerate(shapes):
        X = synth.mixture(40 + b, n, d, k, 40.0, 0.5)
        data.append((X, X[:k].copy()))
    probs = to_device(km, data)
    stats = km.run_batched(probs, 40, tol=1e-300, precision="bf16")
    for (X, C0), st in zip(data, stats):
        r = ref.run(X, C0.astype(np.float64), 40, tol=1e-300)
        assert st["iters_done"] == r["iters_done"] < 40
        assert st["n_changed"] == 0


def test_batched_repeat_uses_tuned_shape(km):
    data = make_batch(SHAPES[:4], seed0=11)
    p1 = to_device(km, data)
    s1 = km.run_batched(p1, 3, precision="bf16")
    p2 = to_device(km, data)
    s2 = km.run_batched(p2, 3, precision="bf16")  # same shapes: cached tuning and graph
    for a, b in zip(p1, p2):
        assert (a[2] != b[2]).sum().item() <= 2
    # every instance reports the batch's autotuned shape: chunk width, instance order, row order
    shapes = {st["batch_shape"] for st in s1 + s2}
    assert len(shapes) == 1
    shape = shapes.pop()
    assert shape % 1000 in (64, 128) and (shape // 1000) % 10 in (0, 1) and shape // 10000 in (0, 1)


def test_batched_errors(km):
    X = torch.randn(100, 200, device=DEV)
    C = X[:4].clone()
    a, s, c = km.alloc_outputs(X, C)
    with pytest.raises(km.KMeansError) as e:
        km.run_batched([(X, C, a, s, c)], 1, precision="bf16")  # d > 128
    assert e.value.status == km.KM_EINVAL
    X = torch.randn(100, 20, device=DEV)
    C = X[:4].clone()
    a, s, c = km.alloc_outputs(X, C)
    with pytest.raises(km.KMeansError) as e:
        km.run_batched([(X, C, a, s, c)], 1, precision="fp32")
    assert e.value.status == km.KM_EUNSUPPORTED
    with pytest.raises(km.KMeansError) as e:
        km.run_batched([(X, C, a, s, c)], 1, precision="bf16x3")
    assert e.value.status == km.KM_EUNSUPPORTED


@pytest.mark.parametrize("shape", ["128,0,1", "64,1,1", "128,1,0", "64,0,0"])
@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_batched_launch_shapes_sorted_steps_parity(km, ref, monkeypatch, shape, precision):
    """Every launch shape the autotuner may pick gives oracle parity, including the steps whose
    tiles run in cluster-sorted order (the second step of a call on, for instances whose k spans
    several chunks). A 2-step run gives the centroids the third step of a 3-step run assigns with
    (the reduce's order can change them by an ulp, within the near-tie and centroid tolerances)."""
    monkeypatch.setenv("KM_BATCH_SHAPE", shape)
    data = make_batch(SHAPES, seed0=2100)
    probs = to_device(km, data)
    km.run_batched(probs, 2, precision=precision)
    C_ins = [p[1].cpu().numpy().astype(np.float64) for p in probs]
    for (X, C0), p in zip(data, probs):
        p[1].copy_(torch.from_numpy(C0).to(DEV))
    stats = km.run_batched(probs, 3, precision=precision)
    for (X, _), (Xd, Cd, a, s, c), C_in, st in zip(data, probs, C_ins, stats):
        ag = a.cpu().numpy()
        assert st["iters_done"] == 3
        assert st["batch_shape"] == int(shape.split(",")[0]) + 1000 * int(shape.split(",")[1]) + \
            10000 * int(shape.split(",")[2])
        parity.check_assign(ref, X, C_in, ag)
        # (an empty cluster keeps the 3-step run's own second-step centroid, equal to C_in up to
        # the reduce order: within the centroid tolerance of the row's magnitude)
        parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), s.cpu().numpy(), c.cpu().numpy(),
                            empty_rtol=parity.CENTROID_TOL)
        parity.check_objective(ref, X, C_in, ag, st["objective"])


def test_batched_launch_shape_knob_rejects_bad_values(km, monkeypatch):
    monkeypatch.setenv("KM_BATCH_SHAPE", "96,0,1")
    probs = to_device(km, make_batch(SHAPES[:2]))
    with pytest.raises(RuntimeError, match="KM_BATCH_SHAPE"):
        km.run_batched(probs, 1, precision="bf16")


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_batched_divide_correctly_rounded(km, precision):
    """The divide rounds each FP64 quotient sum / count correctly and then to FP32 (the reciprocal
    of each count once, then Markstein's correction step). Integer-valued points keep every
    cluster sum exact, so every new coordinate must equal float32(float64(sum) / count) bit for bit."""
    shapes = [(20000, 8, 300), (12000, 32, 7), (9000, 64, 150), (15000, 128, 40), (5000, 3, 1)]
    data = []
    for b, (n, d, k) in enumerate(shapes):
        X = np.clip(np.rint(synth.mixture(7700 + b, n, d, k, 10.0, 1.0) * 25.0), -500, 500).astype(np.float32)
        data.append((X, X[:k].copy()))
    probs = to_device(km, data)
    km.run_batched(probs, 1, precision=precision)
    for (X, C0), (Xd, Cd, a, s, c) in zip(data, probs):
        ag = a.cpu().numpy().astype(np.int64)
        k, d = C0.shape
        cnt = np.bincount(ag, minlength=k)
        assert np.array_equal(c.cpu().numpy(), cnt)
        S = np.zeros((k, d))
        np.add.at(S, ag, X.astype(np.float64))
        assert np.abs(S).max() < 2.0 ** 24  # exact in every partial
        nz = cnt > 0
        want = (S[nz] / cnt[nz, None]).astype(np.float32)
        got = Cd.cpu().numpy()[nz]
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), int((got != want).sum())
        assert np.array_equal(s.cpu().numpy(), S.astype(np.float32))


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_batched_instance_with_more_clusters_than_the_shared_histogram(km, ref, precision):
    """An instance with k > 8192 is counted and scattered with warp-aggregated global atomics
    (the others with shared-memory histograms); one warm step of the batch against the oracle."""
    shapes = [(20000, 8, 9000), (3000, 16, 50), (4000, 64, 300)]
    data = make_batch(shapes, seed0=5100)
    probs = to_device(km, data)
    km.run_batched(probs, 1, precision=precision)
    C_ins = [p[1].cpu().numpy().astype(np.float64) for p in probs]
    stats = km.run_batched(probs, 1, precision=precision, warm_start=True)
    for (X, _), (Xd, Cd, a, s, c), C_in, st in zip(data, probs, C_ins, stats):
        ag = a.cpu().numpy()
        parity.check_assign(ref, X, C_in, ag)
        parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), s.cpu().numpy(), c.cpu().numpy())
        parity.check_objective(ref, X, C_in, ag, st["objective"])


def test_batched_alternating_batches_parity(km, ref):
    """Two batches of the same shapes (so the same tuned launch shape) on different tensors,
    run A, B, A: each call must use its own instance tables and tensor maps."""
    shapes = SHAPES[:5]
    data_a, data_b = make_batch(shapes, seed0=2100), make_batch(shapes, seed0=2200)
    pa, pb = to_device(km, data_a), to_device(km, data_b)
    ba, bb = km.Batch(pa), km.Batch(pb)
    for batch, data, probs in ((ba, data_a, pa), (bb, data_b, pb), (ba, data_a, pa)):
        C_ins = [p[1].cpu().numpy().astype(np.float64) for p in probs]
        stats = batch.run(1, precision="bf16")
        for (X, _), (Xd, Cd, a, s, c), C_in, st in zip(data, probs, C_ins, stats):
            ag = a.cpu().numpy()
            parity.check_assign(ref, X, C_in, ag)
            parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), s.cpu().numpy(), c.cpu().numpy())
            parity.check_objective(ref, X, C_in, ag, st["objective"])


def test_batched_nonfinite_restores_every_c(km, ref):
    """A NaN in one instance's X fails the whole call with KM_ENONFINITE and puts every
    instance's C back to its value on entry; the next clean call is unaffected."""
    shapes = [(1000, 8, 4), (2000, 32, 40), (1500, 64, 300)]
    data = make_batch(shapes, seed0=2300)
    probs = to_device(km, data)
    X1 = probs[1][0]
    keep = X1[17, 5].item()
    X1[17, 5] = float("nan")
    before = [p[1].clone() for p in probs]
    with pytest.raises(km.KMeansError) as e:
        km.run_batched(probs, 3, precision="bf16")
    assert e.value.status == km.KM_ENONFINITE
    for p, c0 in zip(probs, before):
        assert torch.equal(p[1], c0), "C must hold its value on entry after an error"
    X1[17, 5] = keep
    stats = km.run_batched(probs, 1, precision="bf16")
    for (X, C0), (Xd, Cd, a, s, c), st in zip(data, probs, stats):
        C_in = C0.astype(np.float64)
        ag = a.cpu().numpy()
        parity.check_assign(ref, X, C_in, ag)
        parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), s.cpu().numpy(), c.cpu().numpy())
