"""SPADE density downsampling on the GPU (kmeans_spade_densities) against the FP64 oracle.

Every output is an integer decided by FP64 threshold tests, so the comparison is
exact: densities, counts of the evaluated rows and the evaluated-row flags must
equal the oracle's sequential loop element by element.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
POLICY = {"last": 0, "first": 1}


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans

    return kmeans


def widths_for(X, rng, sample=200):
    """apprx = 1.5 x the median nearest-neighbour L1 distance of a row sample, kernel = 10/3 x apprx
    (the ratio of the two widths printed in the paper's generated code)."""
    X64 = X.astype(np.float64)
    rows = rng.choice(X.shape[0], min(sample, X.shape[0]), replace=False)
    nn = []
    for i in rows:
        D = np.abs(X64 - X64[i]).sum(axis=1)
        D[i] = np.inf
        if np.isfinite(D.min()):
            nn.append(D.min())
    a = 1.5 * float(np.median(nn)) if nn else 1.0
    return a, a * 22.29675987 / 6.689027961


def check(km, ref, X, apprx, kernel, policy, Xd=None):
    Xd = torch.from_numpy(X).to(DEV) if Xd is None else Xd
    dens, counts, proc, st = km.spade_densities(Xd, apprx, kernel, policy=policy)
    rd, rc, rp = ref.spade(X, apprx, kernel, POLICY[policy])
    dens, counts, proc = dens.cpu().numpy(), counts.cpu().numpy(), proc.cpu().numpy()
    assert np.array_equal(proc, rp), np.flatnonzero(proc != rp)[:10]
    assert np.array_equal(counts, rc), np.flatnonzero(counts != rc)[:10]
    assert np.array_equal(dens, rd), np.flatnonzero(dens != rd)[:10]
    assert st["n_evaluated"] == int(rp.sum())
    assert st["n_computed"] >= st["n_evaluated"]
    return st


@pytest.mark.parametrize("policy", ["last", "first"])
@pytest.mark.parametrize("n,d,m", [(1, 1, 1), (2, 3, 1), (127, 5, 3), (128, 16, 4), (129, 16, 4), (1000, 13, 8),
                                   (3000, 24, 12), (4099, 33, 20), (2500, 100, 6), (5000, 4, 30)])
def test_matches_oracle(km, ref, n, d, m, policy):
    X = synth.mixture(700 + n + d, n, d, m, 10.0, 0.6)
    apprx, kernel = widths_for(X, np.random.default_rng(n))
    check(km, ref, X, apprx, kernel, policy)


@pytest.mark.parametrize("policy", ["last", "first"])
def test_distances_equal_to_the_widths(km, ref, policy):
    """Integer rows: many L1 distances equal a width exactly, so the FP64 band decides them."""
    rng = np.random.default_rng(5)
    X = rng.integers(-3, 4, (3000, 6)).astype(np.float32)
    st = check(km, ref, X, 4.0, 9.0, policy)
    assert st["n_exact"] > 0
    check(km, ref, X, 9.0, 4.0, policy)  # apprx wider than kernel (the policies' counts differ)


def test_duplicates_and_unaligned_rows(km, ref):
    rng = np.random.default_rng(6)
    base = rng.normal(size=(300, 6)).astype(np.float32)
    X = base[rng.integers(0, 300, 2000)]  # every row repeated several times
    for policy in ("last", "first"):
        check(km, ref, X, 0.5, 3.0, policy)
    # rows that do not start on 16-byte boundaries (4-byte staging path)
    Xall = np.ascontiguousarray(np.concatenate([np.zeros((1, 6), np.float32), X]))
    Xd = torch.from_numpy(Xall).to(DEV)[1:]
    assert Xd.data_ptr() % 16 != 0 and Xd.is_contiguous()
    check(km, ref, X, 0.5, 3.0, "last", Xd=Xd)


def test_found_list_overflow_path(km, ref):
    """apprx wider than every distance: each of the first batch's 1024 candidates finds all
    10,000 rows (more than the found-row list holds), so the evaluated candidates record
    their rows by a second tile pass."""
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (10000, 4)).astype(np.float32)
    st = check(km, ref, X, 100.0, 2.0, "last")
    assert st["overflow_batches"] >= 1 and st["n_evaluated"] == 1
    check(km, ref, X, 100.0, 2.0, "first")


def test_errors_then_usable(km, ref):
    X = torch.zeros(100, 4, device=DEV)
    for a, w in ((0.0, 1.0), (1.0, -1.0), (float("inf"), 1.0), (float("nan"), 1.0)):
        with pytest.raises(km.KMeansError) as e:
            km.spade_densities(X, a, w)
        assert e.value.status == km.KM_EINVAL
    X[3, 2] = float("nan")
    with pytest.raises(km.KMeansError) as e:
        km.spade_densities(X, 1.0, 2.0)
    assert e.value.status == km.KM_ENONFINITE
    X[3, 2] = 0.0
    dens, counts, proc, st = km.spade_densities(X, 1.0, 2.0)
    assert st["n_evaluated"] == 1 and bool((dens == 100).all())


@pytest.mark.slow
def test_full_size_workload(km, ref):
    """The 235,000 x 16 downsampling workload: the whole result against the oracle's
    sequential loop (policy last), and sampled rows of policy first against per-row
    oracle checks (count, first evaluated row within apprx_width)."""
    w = synth.SPADE_WORKLOADS["spade_n235k_d16"]
    X = synth.spade_data(w)
    Xd = torch.from_numpy(X).to(DEV)
    check(km, ref, X, w.apprx, w.kernel, "last", Xd=Xd)
    dens, counts, proc, st = km.spade_densities(Xd, w.apprx, w.kernel, policy="first")
    dens, counts, proc = dens.cpu().numpy(), counts.cpu().numpy(), proc.cpu().numpy()
    cw = max(w.apprx, w.kernel)
    for i in np.random.default_rng(8).choice(w.n, 64, replace=False):
        first, _ = ref.spade_cover(X, int(i), w.apprx, proc)
        assert first >= 0 and (first == i) == bool(proc[i])  # evaluated exactly when no earlier evaluated row finds it
        assert dens[i] == ref.spade_count(X, first, cw)       # the first writer's count
        if proc[i]:
            assert counts[i] == dens[i]
