"""The re-check orders two candidates exactly once their distances differ by a
relative 1e-6 (the near-tie threshold of the parity checks): points built with
two nearly equidistant centroids, relative gaps of 1.05e-6 .. 8e-6 in exact
(FP64) arithmetic on the FP32 inputs, so every precision's margin flags them,
must get the exact argmin, whichever index is the closer one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans

    return kmeans


def exact_d2(X, C):
    X64, C64 = X.astype(np.float64), C.astype(np.float64)
    return ((X64[:, None, :] - C64[None, :, :]) ** 2).sum(-1)


def near_gap_problem(d, pairs, seed):
    """Two points per centroid pair, each pair in its own far-away region; returns X, C and
    the accepted points' exact relative gaps."""
    rng = np.random.default_rng(seed)
    X, C = [], []
    for p in range(pairs):
        o = rng.normal(size=d) * 200.0
        for _ in range(1000):
            x = (o + rng.normal(size=d)).astype(np.float32)
            u1, u2 = rng.normal(size=d), rng.normal(size=d)
            u1 /= np.linalg.norm(u1)
            u2 /= np.linalg.norm(u2)
            g = rng.uniform(1.5e-6, 5e-6)
            ca = (x + 3.0 * u1).astype(np.float32)
            cb = (x + 3.0 * np.sqrt(1.0 + g) * u2).astype(np.float32)
            if rng.random() < 0.5:
                ca, cb = cb, ca  # the closer centroid has the higher index half of the time
            # a second point of the pair: the mirror image through the pair's midpoint keeps a near tie
            x2 = (ca.astype(np.float64) + cb.astype(np.float64) - x.astype(np.float64)).astype(np.float32)
            D = exact_d2(np.stack([x, x2]), np.stack([ca, cb]))
            gaps = np.abs(D[:, 0] - D[:, 1]) / D.max(axis=1)
            if np.all((gaps >= 1.05e-6) & (gaps <= 8e-6)):
                X += [x, x2]
                C += [ca, cb]
                break
        else:
            raise AssertionError("no near-gap point found")
    return np.stack(X), np.stack(C)


@pytest.mark.parametrize("precision,d", [("bf16", 128), ("bf16", 40), ("fp8", 128), ("fp32", 128), ("bf16", 200)])
def test_recheck_orders_gaps_above_threshold(km, precision, d):
    X, C = near_gap_problem(d, 256, seed=7000 + d)
    D = exact_d2(X, C)
    want = D.argmin(axis=1)
    part = np.sort(D, axis=1)
    rel = (part[:, 1] - part[:, 0]) / part[:, 1]
    assert rel.min() >= 1.05e-6 and rel.max() <= 8e-6  # every point is a near tie above the threshold
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(C).to(DEV)
    a, s, c = km.alloc_outputs(Xd, Cd)
    out = km.step(Xd, Cd, a, s, c, precision=precision)
    got = out.assign.cpu().numpy()
    assert np.array_equal(got, want), f"{(got != want).sum()} of {len(want)} points misassigned"
    if precision != "fp32":
        assert out.stats["n_flagged"] == len(want)  # all of them went through the re-check
