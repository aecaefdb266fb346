"""Pins of the oracle's SPADE downsampling (Sec. 4.1) to facts that do not come
from the oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError when
the oracle disagrees with:
  - the hand-worked examples in ``tests/golden/spade_*.txt``,
  - a second, set-based characterisation of the loop evaluated by brute force
    with exact integer arithmetic: the evaluated rows are the greedy set P
    (row i is in P exactly when no row of P before i lies within apprx_width
    of it), and a row's density is the count of the LAST (policy 0, overwriting
    bulk update) or FIRST (policy 1, fill-if-zero) row of P within apprx_width,
  - special cases with closed answers (apprx wider than every distance, apprx
    below every distance, kernel wider than every distance),
  - integer brute force of the per-row helpers (count, cover).
``test_oracle_spade.py`` also runs them against broken builds of the oracle.
"""
from __future__ import annotations

import glob
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_golden(path):
    out = {"cases": []}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split(":", 1))
            vals = val.split()
            if key == "d":
                out["d"] = int(vals[0])
            elif key in ("apprx", "kernel"):
                out[key] = Fraction(vals[0])
            elif key == "X":
                out["X"] = [Fraction(v) for v in vals]
            elif key == "policy":
                out["cases"].append({"policy": int(vals[0])})
            else:
                out["cases"][-1][key] = [int(v) for v in vals]
    return out


def pin_golden(orc):
    files = sorted(glob.glob(os.path.join(GOLDEN, "spade_*.txt")))
    assert len(files) >= 4
    for path in files:
        g = parse_golden(path)
        d = g["d"]
        X = np.array([float(v) for v in g["X"]], np.float32).reshape(-1, d)
        assert all(Fraction(float(v)) == v for v in g["X"]), "golden values must be exact in FP32"
        for case in g["cases"]:
            dens, counts, proc = orc.spade(X, float(g["apprx"]), float(g["kernel"]), case["policy"])
            name = f"{os.path.basename(path)} policy {case['policy']}"
            assert dens.tolist() == case["dens"], (name, dens.tolist())
            assert counts.tolist() == case["counts"], (name, counts.tolist())
            assert proc.tolist() == case["processed"], (name, proc.tolist())


def set_formulation(Xi, apprx, kernel, policy):
    """Densities by the set characterisation, exact: Xi is an integer array, widths Fractions."""
    n = Xi.shape[0]
    D = np.abs(Xi[:, None, :] - Xi[None, :, :]).sum(axis=2)  # exact integers
    near = [[Fraction(int(D[i, j])) < apprx for j in range(n)] for i in range(n)]
    cw = kernel if policy == 0 else max(apprx, kernel)
    cnt = [sum(Fraction(int(D[i, j])) < cw for j in range(n)) for i in range(n)]
    P = []
    for i in range(n):
        if not any(near[p][i] for p in P):
            P.append(i)
    inP = set(P)
    dens, counts, proc = [], [], []
    for i in range(n):
        cover = [p for p in P if near[p][i]]
        q = cover[-1] if policy == 0 else cover[0]
        dens.append(cnt[q])
        counts.append(cnt[i] if i in inP else -1)
        proc.append(1 if i in inP else 0)
    return dens, counts, proc


def pin_set_formulation(orc, trials: int = 300, seed: int = 11):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(1, 13))
        d = int(rng.integers(1, 4))
        Xi = rng.integers(-4, 5, (n, d)).astype(np.int64)
        # widths on the integer grid (distances equal to a width test the strict <) or half-way
        apprx = Fraction(int(rng.integers(1, 9)), int(rng.choice([1, 2])))
        kernel = Fraction(int(rng.integers(1, 13)), int(rng.choice([1, 2])))
        for policy in (0, 1):
            want = set_formulation(Xi, apprx, kernel, policy)
            got = orc.spade(Xi.astype(np.float32), float(apprx), float(kernel), policy)
            assert [g.tolist() for g in got] == [list(w) for w in want], (Xi.tolist(), apprx, kernel, policy)


def pin_special_cases(orc, seed: int = 12):
    rng = np.random.default_rng(seed)
    X = rng.integers(-50, 51, (40, 3)).astype(np.float32)
    n = X.shape[0]
    Di = np.abs(X[:, None, :].astype(np.int64) - X[None, :, :].astype(np.int64)).sum(axis=2)
    for policy in (0, 1):
        # apprx wider than every distance: row 0 alone is evaluated and every density is its count
        dens, counts, proc = orc.spade(X, float(Di.max()) + 1.0, 7.0, policy)
        c0 = int((Di[0] < (7.0 if policy == 0 else Di.max() + 1.0)).sum())
        assert proc.tolist() == [1] + [0] * (n - 1) and (dens == c0).all() and counts[0] == c0
        # kernel wider than every distance: every evaluated row counts all n rows
        dens, counts, proc = orc.spade(X, 5.0, float(Di.max()) + 1.0, policy)
        assert (counts[proc == 1] == n).all() and (dens == n).all()
    # apprx below every nonzero distance and distinct rows: every row is evaluated, densities = counts
    Xd = np.unique(X, axis=0)
    Dd = np.abs(Xd[:, None, :].astype(np.int64) - Xd[None, :, :].astype(np.int64)).sum(axis=2)
    for policy in (0, 1):
        dens, counts, proc = orc.spade(Xd, 0.5, 30.0, policy)
        assert proc.all() and np.array_equal(dens, counts)
        assert np.array_equal(counts, (Dd < 30).sum(axis=1))


def pin_count_cover(orc, seed: int = 13):
    rng = np.random.default_rng(seed)
    X = rng.integers(-9, 10, (300, 5)).astype(np.float32)
    Di = np.abs(X[:, None, :].astype(np.int64) - X[None, :, :].astype(np.int64)).sum(axis=2)
    proc = (rng.random(300) < 0.3).astype(np.uint8)
    for i in (0, 1, 150, 299):
        for w in (0.5, 10.0, 10.5, 40.0):
            assert orc.spade_count(X, i, w) == int((Di[i] < w).sum())
        for a in (3.0, 12.0, 12.5):
            idx = np.flatnonzero((Di[i] < a) & (proc == 1))
            want = (int(idx[0]), int(idx[-1])) if idx.size else (-1, -1)
            assert orc.spade_cover(X, i, a, proc) == want


ALL_PINS = [pin_golden, pin_set_formulation, pin_special_cases, pin_count_cover]
