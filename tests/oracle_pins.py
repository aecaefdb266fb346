"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError when
the oracle disagrees with:
  - the hand-worked examples in ``tests/golden/`` (exact rationals),
  - exhaustive enumeration of every assignment vector on tiny inputs, with exact
    rational arithmetic (the Lloyd assignment minimises J(a, C) over a),
  - the least-squares property of the update (the member mean zeroes the
    gradient of J over c and no perturbation lowers J),
  - closed forms (k = 1, k = n, sorted 1-D data) and library routines
    (numpy mean/var, torch.cdist),
  - invariants of any run (counts sum to n, monotone objective, permutation
    equivariance, resumability).
The same functions run against deliberately broken builds of the oracle
(``test_oracle.py``) to show that they catch plausible mistakes.
"""
from __future__ import annotations

import glob
import itertools
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_golden(path):
    d = None
    X = C0 = None
    steps = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split(":", 1))
            vals = val.split()
            if key == "d":
                d = int(vals[0])
            elif key == "X":
                X = [Fraction(v) for v in vals]
            elif key == "C0":
                C0 = [Fraction(v) for v in vals]
            elif key == "step":
                steps.append({})
            elif key in ("assign", "counts"):
                steps[-1][key] = [int(v) for v in vals]
            elif key == "C":
                steps[-1][key] = [Fraction(v) for v in vals]
            elif key == "J":
                steps[-1][key] = Fraction(vals[0])
    return d, X, C0, steps


def golden_files():
    return sorted(glob.glob(os.path.join(GOLDEN, "lloyd_*.txt")))


def _close(a: float, b: Fraction, rel: float = 1e-14, abs_: float = 1e-14) -> bool:
    return abs(Fraction(a) - b) <= max(abs_, rel * abs(b))


def pin_golden(orc):
    files = golden_files()
    assert len(files) >= 4
    for path in files:
        d, Xf, C0f, steps = parse_golden(path)
        X = np.array([float(v) for v in Xf], np.float32).reshape(-1, d)
        assert all(Fraction(float(v)) == v for v in Xf), "fixture X must be exact in FP32"
        C = np.array([float(v) for v in C0f], np.float64).reshape(-1, d)
        for s, exp in enumerate(steps):
            r = orc.step(X, C)
            assert r["assign"].tolist() == exp["assign"], (path, s, "assign")
            assert r["counts"].tolist() == exp["counts"], (path, s, "counts")
            assert all(_close(a, b) for a, b in zip(r["C"].ravel().tolist(), exp["C"])), (path, s, "C")
            assert _close(r["objective"], exp["J"]), (path, s, "J", r["objective"], exp["J"])
            C = r["C"]
        # a multi-step run reaches the same state as the chained single steps
        rr = orc.run(X, np.array([float(v) for v in C0f]).reshape(-1, d), len(steps))
        assert rr["assign"].tolist() == steps[-1]["assign"], (path, "run assign")
        assert all(_close(a, b) for a, b in zip(rr["C"].ravel().tolist(), steps[-1]["C"]))
        assert all(_close(j, e["J"]) for j, e in zip(rr["objectives"].tolist(), steps))


def _exact_sqdist(x, c):
    return sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, c))


def pin_bruteforce_assign(orc, trials: int = 150, seed: int = 1):
    """Enumerate every assignment vector a in [k]^n with exact rationals."""
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(1, 7))
        k = int(rng.integers(1, min(3, n) + 1))
        d = int(rng.integers(1, 4))
        X = rng.integers(-3, 4, size=(n, d)).astype(np.float32)
        C = (rng.integers(-6, 7, size=(k, d)) / 2.0).astype(np.float64)
        if rng.random() < 0.3:  # force duplicate centroids now and then
            C[-1] = C[0]
        D = [[_exact_sqdist(X[i], C[j]) for j in range(k)] for i in range(n)]
        best_J, minimisers = None, []
        for a in itertools.product(range(k), repeat=n):
            J = sum(D[i][a[i]] for i in range(n))
            if best_J is None or J < best_J:
                best_J, minimisers = J, [a]
            elif J == best_J:
                minimisers.append(a)
        canonical = min(minimisers)  # lexicographically smallest = lowest index per point
        a, dmin, gap, second = orc.assign(X, C)
        assert tuple(a.tolist()) == canonical, (X.tolist(), C.tolist(), a.tolist(), canonical)
        assert tuple(a.tolist()) in minimisers
        for i in range(n):
            assert Fraction(float(dmin[i])) == D[i][a[i]]
            if k > 1:
                rest = sorted((D[i][j], j) for j in range(k) if j != a[i])
                d2 = rest[0][0]
                assert int(second[i]) == rest[0][1]
                exp_gap = (d2 - D[i][a[i]]) / d2 if d2 > 0 else Fraction(0)
                assert abs(Fraction(float(gap[i])) - exp_gap) <= Fraction(1, 10**14)
            else:
                assert np.isinf(gap[i])
        r = orc.step(X, C)
        assert _close(r["objective"], best_J, rel=1e-15), (r["objective"], best_J)


def pin_update_least_squares(orc, trials: int = 60, seed: int = 2):
    """The update zeroes sum_{a_i=j}(x_i - c_j) exactly and no perturbation lowers J."""
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(1, 9))
        k = int(rng.integers(1, 4))
        d = int(rng.integers(1, 4))
        X = rng.integers(-5, 6, size=(n, d)).astype(np.float32)
        a = rng.integers(0, k, size=n).astype(np.int32)
        Cprev = (rng.integers(-8, 9, size=(k, d)) / 4.0).astype(np.float64)
        sums, counts, Cnew = orc.update(X, a, Cprev)
        assert counts.sum() == n
        for j in range(k):
            members = [i for i in range(n) if a[i] == j]
            assert counts[j] == len(members)
            if not members:
                assert np.array_equal(Cnew[j], Cprev[j]), "empty cluster keeps its centroid"
                assert np.all(sums[j] == 0)
                continue
            for t in range(d):
                assert Fraction(float(sums[j, t])) == sum(Fraction(float(X[i, t])) for i in members)
                # gradient of sum_i (x_it - c)^2 at c = Cnew_jt is ~0 (up to one rounding of c)
                g = sum(Fraction(float(X[i, t])) - Fraction(float(Cnew[j, t])) for i in members)
                assert abs(g) <= len(members) * abs(Fraction(float(Cnew[j, t]))) * Fraction(2, 2**52) + Fraction(1, 2**60)

            def Jj(c):
                return sum(_exact_sqdist(X[i], c) for i in members)

            base = Jj(Cnew[j])
            for t in range(d):
                for eps in (0.5, 1e-3):
                    for sgn in (1, -1):
                        c = Cnew[j].copy()
                        c[t] += sgn * eps
                        assert Jj(c) > base


def pin_closed_forms(orc, seed: int = 3):
    rng = np.random.default_rng(seed)
    # k = 1: every point in cluster 0; the centroid is the global mean; J = n * total variance
    X = rng.normal(size=(500, 4)).astype(np.float32) * 3 + 1
    r = orc.step(X, X[:1])
    assert np.all(r["assign"] == 0)
    mean = X.astype(np.float64).mean(axis=0)
    assert np.allclose(r["C"][0], mean, rtol=1e-12, atol=1e-12)
    X64 = X.astype(np.float64)
    Jexp = float(((X64 - X64[0]) ** 2).sum())
    assert abs(r["objective"] - Jexp) <= 1e-9 * Jexp
    r2 = orc.step(X, r["C"])
    Jvar = float(X.astype(np.float64).var(axis=0).sum() * X.shape[0])
    assert abs(r2["objective"] - Jvar) <= 1e-9 * Jvar
    # k = n with distinct points and C0 = X: identity assignment, J = 0, C unchanged
    Xd = rng.permutation(np.arange(40, dtype=np.float32) * 1.5).reshape(20, 2)
    r = orc.step(Xd, Xd)
    assert r["assign"].tolist() == list(range(20))
    assert r["objective"] == 0.0
    assert np.array_equal(r["C"], Xd.astype(np.float64))
    assert np.all(r["counts"] == 1)
    # sorted 1-D data with sorted centroids: clusters are contiguous intervals in order
    x = np.sort(rng.normal(size=300)).astype(np.float32)
    C = np.sort(rng.choice(x, 7, replace=False)).astype(np.float64)
    a, *_ = orc.assign(x, C)
    assert np.all(np.diff(a) >= 0)


def pin_library_crosscheck(orc, seed: int = 4):
    """argmin and top-2 gap against torch.cdist in FP64 on tie-free random data."""
    import torch

    rng = np.random.default_rng(seed)
    for n, d, k in ((257, 3, 5), (300, 17, 33), (64, 40, 64)):
        X = rng.normal(size=(n, d)).astype(np.float32)
        C = rng.normal(size=(k, d)) * 0.9
        D = torch.cdist(torch.from_numpy(X.astype(np.float64)), torch.from_numpy(C)) ** 2
        Ds, idx = torch.sort(D, dim=1, stable=True)
        a, dmin, gap, second = orc.assign(X, C)
        assert np.array_equal(a, idx[:, 0].numpy().astype(np.int32))
        assert np.allclose(dmin, Ds[:, 0].numpy(), rtol=1e-9, atol=1e-9)
        if k > 1:
            assert np.array_equal(second, idx[:, 1].numpy().astype(np.int32))
            g = ((Ds[:, 1] - Ds[:, 0]) / Ds[:, 1]).numpy()
            assert np.allclose(gap, g, rtol=1e-6, atol=1e-9)


def pin_invariants(orc, seed: int = 5):
    import synth

    X = synth.mixture(0xC0FFEE + seed, 3000, 6, 9, 4.0, 1.0)
    C0 = X[:9].astype(np.float64)
    run = orc.run(X, C0, 10)
    J = run["objectives"]
    assert len(J) == 10
    assert np.all(J[1:] <= J[:-1] * (1 + 1e-12)), "Lloyd objective must not increase"
    assert run["counts"].sum() == X.shape[0]
    # 5 + 5 steps equal 10 steps (the whole state is C)
    r5 = orc.run(X, C0, 5)
    r55 = orc.run(X, r5["C"], 5)
    assert np.array_equal(r55["assign"], run["assign"])
    assert np.array_equal(r55["C"], run["C"])
    # each assignment is an argmin of the distances to the centroids it used
    C = C0
    for _ in range(3):
        r = orc.step(X, C)
        D = ((X[:, None, :].astype(np.float64) - C[None, :, :]) ** 2).sum(-1)
        assert np.all(D[np.arange(len(X)), r["assign"]] <= D.min(axis=1))
        means = np.zeros_like(C)
        np.add.at(means, r["assign"], X.astype(np.float64))
        cnt = np.bincount(r["assign"], minlength=C.shape[0])
        nz = cnt > 0
        means[nz] /= cnt[nz, None]
        means[~nz] = C[~nz]
        assert np.allclose(r["C"], means, rtol=1e-12, atol=1e-12)
        C = r["C"]
    # permuting the points permutes the assignment (the loop body runs once per index, in no set order)
    perm = np.random.default_rng(seed).permutation(X.shape[0])
    r1 = orc.step(X, C)
    r2 = orc.step(X[perm], C)
    assert np.array_equal(r2["assign"], r1["assign"][perm])
    assert np.array_equal(r2["counts"], r1["counts"])
    assert np.allclose(r2["C"], r1["C"], rtol=1e-13, atol=1e-13)


def pin_tolerance_stop(orc):
    """tol > 0 stops after the first step whose assignment repeats (example A: step 3)."""
    d, Xf, C0f, steps = parse_golden(os.path.join(GOLDEN, "lloyd_1d_example_a.txt"))
    X = np.array([float(v) for v in Xf], np.float32).reshape(-1, d)
    C0 = np.array([float(v) for v in C0f]).reshape(-1, d)
    r = orc.run(X, C0, 50, tol=1e-300)
    assert r["iters_done"] == 3, r["iters_done"]
    r = orc.run(X, C0, 50, tol=1e6)  # every shift is below a huge tolerance: one step
    assert r["iters_done"] == 1


ALL_PINS = [pin_golden, pin_bruteforce_assign, pin_update_least_squares, pin_closed_forms,
            pin_library_crosscheck, pin_invariants, pin_tolerance_stop]
