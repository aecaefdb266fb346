"""The seeded generator: determinism, row independence, and the mixture's moments."""
import numpy as np

import synth
from synth import WORKLOADS


def test_deterministic_and_row_independent():
    a = synth.mixture(123, 1000, 7, 5, 3.0, 0.5)
    b = synth.mixture(123, 1000, 7, 5, 3.0, 0.5)
    assert np.array_equal(a, b)
    part = synth.mixture(123, 100, 7, 5, 3.0, 0.5, row0=450)
    assert np.array_equal(part, a[450:550])
    assert not np.array_equal(a, synth.mixture(124, 1000, 7, 5, 3.0, 0.5))


def test_splitmix64_reference_values():
    # Published SplitMix64 outputs for the seed 1234567 (Steele, Lea, Flood 2014 reference code)
    assert synth.splitmix64(1234567, 0) == 6457827717110365317
    assert synth.splitmix64(1234567, 1) == 3203168211198807973


def test_mixture_moments():
    X, comp = synth.mixture(7, 200_000, 3, 4, 5.0, 0.7, with_comp=True)
    mu = synth.means(7, 4, 3, 5.0)
    assert np.all(np.abs(mu) <= 5.0)
    assert set(np.unique(comp)) == {0, 1, 2, 3}
    resid = X.astype(np.float64) - mu[comp]
    assert abs(resid.mean()) < 0.01
    assert abs(resid.std() - 0.7) < 0.01
    frac = np.bincount(comp) / len(comp)
    assert np.all(np.abs(frac - 0.25) < 0.01)


def test_uniform_in_open_interval():
    u = np.array([synth.u01(1, 2, i) for i in range(2000)])
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.02


def test_batched_shapes_in_range():
    from synth import batched_instances

    inst = batched_instances()
    assert len(inst) == 512
    for w in inst:
        assert 1000 <= w.n <= 200_000 and w.d in (8, 32, 64, 128) and 4 <= w.k <= 512
    assert len({w.d for w in inst}) == 4


def test_workload_table():
    w = WORKLOADS["fp32_n1M_d64_k256"]
    assert (w.n, w.d, w.k, w.iters) == (1 << 20, 64, 256, 20)
    assert w.flops_per_iter == 2.0 * (1 << 20) * 256 * 64
